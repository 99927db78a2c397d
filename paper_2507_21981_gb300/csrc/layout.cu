// Storage order of a node's Gaussians: Morton (Z-order) over the node's bounding box.
//
// Sec. III-B ("Asset Formatting"): every asset is converted once into the renderer's own
// format before simulation.  The renderer processes a node in chunks of 32 consecutive
// Gaussians and culls a whole chunk per view with one bounding-sphere test; that test rejects
// work only when consecutive Gaussians are close in space, which an arbitrary training order
// does not give.  Sorting the Gaussians along a Z-order curve of their means does.  The order
// is a host-side preprocessing step the caller applies to its own arrays (all attributes
// permuted alike); the rendered image is that of the permuted node, whose global ids follow the
// new order.
#include <algorithm>
#include <cmath>
#include <utility>
#include <vector>

#include "dgs.h"

namespace {

// Spreads the low 21 bits of x so that bit i lands at bit 3i.
uint64_t spread3(uint64_t x) {
    x &= 0x1fffffull;
    x = (x | (x << 32)) & 0x1f00000000ffffull;
    x = (x | (x << 16)) & 0x1f0000ff0000ffull;
    x = (x | (x << 8)) & 0x100f00f00f00f00full;
    x = (x | (x << 4)) & 0x10c30c30c30c30c3ull;
    x = (x | (x << 2)) & 0x1249249249249249ull;
    return x;
}

}  // namespace

extern "C" int dgs_spatial_order(const float* mean, int64_t n, int64_t* perm) {
    if (n < 0 || (n > 0 && (!mean || !perm))) return DGS_ERR_INVALID_ARG;
    if (n == 0) return DGS_OK;
    double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int64_t i = 0; i < n; ++i) {
        const float* m = mean + 3 * i;
        if (!(std::isfinite(m[0]) && std::isfinite(m[1]) && std::isfinite(m[2]))) continue;
        for (int a = 0; a < 3; ++a) {
            lo[a] = std::min(lo[a], (double)m[a]);
            hi[a] = std::max(hi[a], (double)m[a]);
        }
    }
    // one scale for all axes keeps the cells cubic
    double ext = 0.0;
    for (int a = 0; a < 3; ++a) ext = std::max(ext, hi[a] - lo[a]);
    const double scale = ext > 0.0 ? (double)((1u << 21) - 1u) / ext : 0.0;
    std::vector<std::pair<uint64_t, int64_t>> key((size_t)n);
    for (int64_t i = 0; i < n; ++i) {
        const float* m = mean + 3 * i;
        uint64_t code = ~0ull;   // non-finite means go last
        if (std::isfinite(m[0]) && std::isfinite(m[1]) && std::isfinite(m[2])) {
            uint64_t q[3];
            for (int a = 0; a < 3; ++a) {
                const double t = std::floor(((double)m[a] - lo[a]) * scale);
                q[a] = (uint64_t)std::min(std::max(t, 0.0), (double)((1u << 21) - 1u));
            }
            code = spread3(q[0]) | (spread3(q[1]) << 1) | (spread3(q[2]) << 2);
        }
        key[(size_t)i] = {code, i};
    }
    std::sort(key.begin(), key.end());   // ties by index: deterministic
    for (int64_t i = 0; i < n; ++i) perm[i] = key[(size_t)i].second;
    return DGS_OK;
}
