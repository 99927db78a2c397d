// Stable LSD radix sort of (64-bit key, 32-bit value) pairs in the onesweep style (kernel K3).
//
// Sec. III-A: the 3DGS rasterizer orders the (tile, depth) pairs of every view with a fast
// GPU sort before blending.  Keys are (global tile << 28) | depth-key, values the instance
// index; emission in global-id order plus stability breaks equal depths by id.
//
// Structure: one upfront pass builds the 256-bin histograms of every digit at once; then
// each digit is one kernel in which a block takes the next 4096-key partition from an atomic
// counter, ranks its keys by digit inside the block (warp match + per-warp counters), and
// finds its global offset per digit by decoupled look-back over the partitions before it
// (status word = 2-bit flag | 30-bit count).  Only digits inside the significant key bits
// are sorted.  Look-back spins are bounded by a wall-clock limit; on expiry the kernel sets
// kErrTimeout and finishes (the output is then invalid and the host reports it).
#include <algorithm>

#include "dgs_internal.cuh"

namespace dgs {
namespace {

constexpr int kThreads = 256;
constexpr int kItems = 16;
constexpr int kTile = kThreads * kItems;          // 4096 keys per partition
constexpr int kWarps = kThreads / 32;
constexpr uint32_t kFlagAgg = 1u << 30, kFlagInc = 2u << 30, kCountMask = (1u << 30) - 1u;
constexpr uint64_t kSpinLimitNs = 1000000000ull;  // 1 s

__device__ __forceinline__ uint32_t ld_relaxed(const uint32_t* p) {
    uint32_t v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_relaxed(uint32_t* p, uint32_t v) {
    asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ uint32_t live_count(uint32_t n, const uint32_t* d_n) { return d_n ? min(*d_n, n) : n; }

__global__ void __launch_bounds__(kThreads) k_hist(const uint64_t* __restrict__ keys, uint32_t n,
                                                   const uint32_t* __restrict__ d_n, int passes, uint32_t* hist) {
    __shared__ uint32_t sh[8 * 256];
    n = live_count(n, d_n);
    for (int i = threadIdx.x; i < passes * 256; i += kThreads) sh[i] = 0;
    __syncthreads();
    for (uint32_t i = blockIdx.x * kThreads + threadIdx.x; i < n; i += gridDim.x * kThreads) {
        const uint64_t k = keys[i];
        for (int p = 0; p < passes; ++p) atomicAdd(&sh[p * 256 + (uint32_t)((k >> (8 * p)) & 255u)], 1u);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < passes * 256; i += kThreads)
        if (sh[i]) atomicAdd(&hist[i], sh[i]);
}

// one block, 256 threads: exclusive scan of each pass's 256 bins, in place
__global__ void __launch_bounds__(256) k_hist_scan(uint32_t* hist, int passes) {
    __shared__ uint32_t s[256];
    for (int p = 0; p < passes; ++p) {
        const uint32_t x = hist[p * 256 + threadIdx.x];
        s[threadIdx.x] = x;
        __syncthreads();
        for (int o = 1; o < 256; o <<= 1) {
            const uint32_t y = threadIdx.x >= (unsigned)o ? s[threadIdx.x - o] : 0u;
            __syncthreads();
            s[threadIdx.x] += y;
            __syncthreads();
        }
        hist[p * 256 + threadIdx.x] = s[threadIdx.x] - x;
        __syncthreads();
    }
}

__global__ void __launch_bounds__(kThreads) k_onesweep(const uint64_t* __restrict__ kin, const uint32_t* __restrict__ vin,
                                                      uint64_t* __restrict__ kout, uint32_t* __restrict__ vout, uint32_t n,
                                                      const uint32_t* __restrict__ d_n, int shift,
                                                      const uint32_t* __restrict__ digit_off, uint32_t* status,
                                                      uint32_t* counter, uint32_t* err) {
    extern __shared__ __align__(16) unsigned char smem[];
    uint64_t* s_keys = reinterpret_cast<uint64_t*>(smem);                          // kTile
    uint32_t* s_vals = reinterpret_cast<uint32_t*>(smem + kTile * 8);               // kTile
    uint32_t* s_whist = reinterpret_cast<uint32_t*>(smem + kTile * 12);             // kWarps x 256
    __shared__ uint32_t s_dexcl[256];
    __shared__ uint32_t s_gbase[256];
    __shared__ uint32_t s_wsum[kWarps];
    __shared__ uint32_t s_part;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) s_part = atomicAdd(counter, 1u);
    for (int i = tid; i < kWarps * 256; i += kThreads) s_whist[i] = 0;
    __syncthreads();
    const uint32_t part = s_part;
    n = live_count(n, d_n);
    // a capacity-sized grid: partitions past the live count have no keys (and no later
    // partition looks back at them)
    if (part * (uint64_t)kTile >= n && part > 0) return;
    const uint32_t base = part * (uint32_t)kTile;

    uint64_t k[kItems];
    uint32_t v[kItems], rank[kItems];
#pragma unroll
    for (int j = 0; j < kItems; ++j) {
        const uint32_t idx = base + warp * (kItems * 32) + j * 32 + lane;
        if (idx < n) { k[j] = kin[idx]; v[j] = vin[idx]; }
        else { k[j] = ~0ull; v[j] = 0; }
    }
    // rank within the warp, in original order (round j covers 32 consecutive keys)
    const uint32_t lt = (1u << lane) - 1u;
    uint32_t* wh = s_whist + warp * 256;
#pragma unroll
    for (int j = 0; j < kItems; ++j) {
        const uint32_t d = (uint32_t)(k[j] >> shift) & 255u;
        const uint32_t peers = __match_any_sync(0xffffffffu, d);
        const uint32_t pre = wh[d];
        rank[j] = pre + __popc(peers & lt);
        __syncwarp();
        if ((peers & lt) == 0) wh[d] = pre + __popc(peers);
        __syncwarp();
    }
    __syncthreads();
    // thread d: exclusive prefix over warps and the partition total of digit d
    const uint32_t d = tid;
    uint32_t total = 0;
#pragma unroll
    for (int w = 0; w < kWarps; ++w) {
        const uint32_t c = s_whist[w * 256 + d];
        s_whist[w * 256 + d] = total;
        total += c;
    }
    // decoupled look-back over earlier partitions for digit d
    uint32_t excl = 0;
    if (part == 0) {
        st_relaxed(&status[d], kFlagInc | total);
    } else {
        st_relaxed(&status[(size_t)part * 256 + d], kFlagAgg | total);
        int64_t p = (int64_t)part - 1;
        uint64_t t0 = 0;
        uint32_t spins = 0;
        while (p >= 0) {
            const uint32_t s = ld_relaxed(&status[(size_t)p * 256 + d]);
            const uint32_t f = s & ~kCountMask;
            if (f == 0) {
                if ((++spins & 1023u) == 0) {
                    const uint64_t now = global_timer_ns();
                    if (t0 == 0) t0 = now;
                    else if (now - t0 > kSpinLimitNs) { atomicOr(err, kErrTimeout); break; }
                }
                continue;
            }
            excl += s & kCountMask;
            if (f == kFlagInc) break;
            --p;
        }
        st_relaxed(&status[(size_t)part * 256 + d], kFlagInc | (excl + total));
    }
    s_gbase[d] = digit_off[d] + excl;
    // block exclusive scan of the digit totals -> local digit offsets
    {
        uint32_t x = total;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) s_wsum[warp] = x;
        __syncthreads();
        uint32_t wpre = 0;
        for (int w = 0; w < warp; ++w) wpre += s_wsum[w];
        s_dexcl[d] = wpre + x - total;
    }
    __syncthreads();
    // local scatter: digit-major order inside the partition
#pragma unroll
    for (int j = 0; j < kItems; ++j) {
        const uint32_t dj = (uint32_t)(k[j] >> shift) & 255u;
        const uint32_t pos = s_dexcl[dj] + s_whist[warp * 256 + dj] + rank[j];
        s_keys[pos] = k[j];
        s_vals[pos] = v[j];
    }
    __syncthreads();
#pragma unroll 4
    for (int i = tid; i < kTile; i += kThreads) {
        const uint64_t key = s_keys[i];
        const uint32_t dj = (uint32_t)(key >> shift) & 255u;
        const uint32_t g = s_gbase[dj] + (uint32_t)i - s_dexcl[dj];
        if (g < n) { kout[g] = key; vout[g] = s_vals[i]; }
    }
}

}  // namespace

int sort_passes(int key_bits) { return (key_bits + 7) / 8; }

size_t sort_status_words(uint32_t n) { return ((size_t)n + kTile - 1) / kTile * 256; }

void sort_prepare() {
    static bool attr_set = false;
    if (!attr_set) {
        cudaFuncSetAttribute(k_onesweep, cudaFuncAttributeMaxDynamicSharedMemorySize, kTile * 12 + kWarps * 256 * 4);
        attr_set = true;
    }
}

// hist: [8*256] words, counters: [8] words, status: sort_status_words(n) words.
void launch_sort(const Launch& L, uint64_t* keys, uint32_t* vals, uint64_t* keys_alt, uint32_t* vals_alt, uint32_t n,
                 int key_bits, uint32_t* hist, uint32_t* status, uint32_t* counters, uint32_t* err,
                 uint64_t** keys_out, uint32_t** vals_out, float* sort_ms_slot, cudaEvent_t* evs,
                 const uint32_t* d_n) {
    (void)sort_ms_slot; (void)evs;
    *keys_out = keys;
    *vals_out = vals;
    // with a device-side count every pass runs (the output lands in the same buffer whatever
    // the count); a host-known count of 0 or 1 is already sorted
    if (n <= 1 && !d_n) return;
    if (n == 0) return;
    const int passes = sort_passes(key_bits);
    sort_prepare();
    cudaMemsetAsync(hist, 0, sizeof(uint32_t) * 256 * passes, L.stream);
    cudaMemsetAsync(counters, 0, sizeof(uint32_t) * 8, L.stream);
    const int hist_blocks = (int)std::min<uint32_t>(4 * 152, (n + kThreads * 8 - 1) / (kThreads * 8));
    k_hist<<<hist_blocks, kThreads, 0, L.stream>>>(keys, n, d_n, passes, hist);
    k_hist_scan<<<1, 256, 0, L.stream>>>(hist, passes);
    *L.launches += 2;
    const uint32_t parts = (n + kTile - 1) / kTile;
    uint64_t *ki = keys, *ko = keys_alt;
    uint32_t *vi = vals, *vo = vals_alt;
    for (int p = 0; p < passes; ++p) {
        cudaMemsetAsync(status, 0, sizeof(uint32_t) * 256 * (size_t)parts, L.stream);
        k_onesweep<<<parts, kThreads, kTile * 12 + kWarps * 256 * 4, L.stream>>>(ki, vi, ko, vo, n, d_n, 8 * p,
                                                                                 hist + p * 256, status, counters + p,
                                                                                 err);
        ++*L.launches;
        uint64_t* tk = ki; ki = ko; ko = tk;
        uint32_t* tv = vi; vi = vo; vo = tv;
    }
    *keys_out = ki;
    *vals_out = vi;
}

}  // namespace dgs
