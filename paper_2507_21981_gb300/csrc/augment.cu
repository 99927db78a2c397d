// Image randomisation of rendered RGB (Sec. IV: overlay blend, HSV jitter, random gamma) as a
// separate pass over a batch of views, in place.  The compositor applies the same per-pixel
// function in its epilogue when a randomisation is set; this kernel serves images rendered
// without it.
//
// The pass is bound by HBM: 24 bytes of RGB per pixel plus 3 bytes of overlay where the view's
// weight is non-zero.
#include "dgs_internal.cuh"

namespace dgs {
namespace {

constexpr int kThreads = 256;

// Thread = one quad of 4 consecutive output pixels (48 bytes: three 16-byte loads and stores
// when the quad lies inside one view and the buffer is 16-byte aligned; per-pixel scalar
// accesses at view edges).  Lane 0 of each warp finds the view of the warp's first quad.  Quads are enumerated view by view (spans[v].q0 = first quad of
// view v); a view whose first pixel is not a multiple of 4 shares its edge quads with its
// neighbours, each thread touching only its own view's pixels.
__global__ void __launch_bounds__(kThreads) k_augment(const AugSpan* __restrict__ spans, int V, int64_t n_quads,
                                                      const dgs_augment* __restrict__ aug,
                                                      const uint8_t* __restrict__ overlay, int ow, int oh,
                                                      float* __restrict__ rgb, bool vec) {
    const int64_t j0 = (int64_t)blockIdx.x * kThreads + (threadIdx.x & ~31);   // the warp's first quad
    int v = 0;
    if ((threadIdx.x & 31) == 0) {               // view of the warp's first quad
        int lo = 0, hi = V - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (spans[mid].q0 <= j0) lo = mid; else hi = mid - 1;
        }
        v = lo;
    }
    v = __shfl_sync(0xffffffffu, v, 0);
    const int64_t j = (int64_t)blockIdx.x * kThreads + threadIdx.x;
    if (j >= n_quads) return;
    while (v + 1 < V && spans[v + 1].q0 <= j) ++v;
    const AugSpan sp = spans[v];
    const int32_t n = sp.W * sp.H;               // <= 2^30
    const int64_t p0 = (sp.pix_off / 4 + (j - sp.q0)) * 4;
    const int32_t l0 = (int32_t)(p0 - sp.pix_off);   // local index of the quad's first pixel, >= -3
    float* base = rgb + p0 * 3;
    float c[12];
    const bool full = vec && l0 >= 0 && l0 + 4 <= n;
    if (full) {
        const float4* b4 = reinterpret_cast<const float4*>(base);
        const float4 x0 = b4[0], x1 = b4[1], x2 = b4[2];
        c[0] = x0.x; c[1] = x0.y; c[2] = x0.z; c[3] = x0.w;
        c[4] = x1.x; c[5] = x1.y; c[6] = x1.z; c[7] = x1.w;
        c[8] = x2.x; c[9] = x2.y; c[10] = x2.z; c[11] = x2.w;
    } else {
#pragma unroll
        for (int k = 0; k < 4; ++k)
            if (l0 + k >= 0 && l0 + k < n) { c[3 * k] = base[3 * k]; c[3 * k + 1] = base[3 * k + 1]; c[3 * k + 2] = base[3 * k + 2]; }
    }
    const dgs_augment a = aug[v];
    const int32_t lf = max(l0, 0);
    int y = lf / sp.W, x = lf - y * sp.W;
    // overlay column and row of the first pixel, then stepped pixel by pixel
    const bool blend = a.overlay_beta != 0.f;
    int ox = 0, oy = 0;
    if (blend) {
        ox = (a.overlay_x + x) % ow;
        oy = (a.overlay_y + y) % oh;
    }
    const uint8_t* frame = overlay + (int64_t)a.overlay_frame * oh * ow * 3;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        if (l0 + k >= 0 && l0 + k < n) {
            augment_pixel(a, frame + ((int64_t)oy * ow + ox) * 3, c[3 * k], c[3 * k + 1], c[3 * k + 2]);
            if (++x == sp.W) {                   // next row: overlay column back to the crop origin
                x = 0;
                ox = a.overlay_x;
                if (++oy == oh) oy = 0;
            } else if (++ox == ow) {
                ox = 0;
            }
        }
    }
    if (full) {
        float4* b4 = reinterpret_cast<float4*>(base);
        b4[0] = make_float4(c[0], c[1], c[2], c[3]);
        b4[1] = make_float4(c[4], c[5], c[6], c[7]);
        b4[2] = make_float4(c[8], c[9], c[10], c[11]);
    } else {
#pragma unroll
        for (int k = 0; k < 4; ++k)
            if (l0 + k >= 0 && l0 + k < n) { base[3 * k] = c[3 * k]; base[3 * k + 1] = c[3 * k + 1]; base[3 * k + 2] = c[3 * k + 2]; }
    }
}

}  // namespace

void launch_augment(const Launch& L, const AugSpan* spans, int V, int64_t n_quads, const dgs_augment* aug,
                    const uint8_t* overlay, int ow, int oh, float* rgb) {
    if (n_quads <= 0) return;
    const bool vec = (reinterpret_cast<uintptr_t>(rgb) & 15u) == 0;
    const int64_t blocks = (n_quads + kThreads - 1) / kThreads;
    k_augment<<<(unsigned)blocks, kThreads, 0, L.stream>>>(spans, V, n_quads, aug, overlay, ow, oh, rgb, vec);
    ++*L.launches;
}

}  // namespace dgs
