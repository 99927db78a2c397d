// dgs_render_noalloc: the batched render of Sec. III-A / III-C with all of its scratch in one
// fixed, statically allocated device array, for callers that must not allocate GPU memory
// (a deployment variant; the paper has no counterpart).
//
// Who needs it: a host program that runs inside another framework's memory manager (a
// caching allocator that owns the device budget and forbids foreign cudaMalloc calls), a
// control loop that cannot afford the device-wide synchronisation cudaFree and cudaMalloc may
// imply in the middle of a step, or code certified to allocate nothing after start-up.  Such
// a caller still passes its own inputs and outputs; everything else the render needs (tables,
// counters, projected records, sort buffers, tile ranges) is carved out of g_scratch.
//
// Limits and sharing: g_scratch is kScratchBytes (64 MiB) on every device that loads the
// library, held until the process exits.  A batch whose tables or tile pairs do not fit is
// rejected with DGS_ERR_CAPACITY before any kernel is queued for its second phase.  Every
// call on a device uses the same array and leaves its contents behind; the call clears what
// must start at zero (error word, histograms, counters, look-back status, tile ranges).  Two
// calls whose work overlaps on the GPU (different streams, or different host threads) race
// on the array and corrupt each other's results: serialise them.
//
// Set-up: the device address of g_scratch is resolved once per device, by the first call
// made with that device current (cudaGetSymbolAddress); make that first call before any
// stream capture begins on the device.
#include <algorithm>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "dgs_internal.cuh"

using namespace dgs;

namespace {

constexpr size_t kScratchBytes = 64ull << 20;
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
void* g_scratch_dev[kMaxDevices] = {};
std::mutex g_scratch_mu;

// Device address of g_scratch on the current device (resolved once per device).
cudaError_t scratch_address(unsigned char** out) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_scratch_mu);
    if (!g_scratch_dev[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_dev[dev] = p;
    }
    *out = static_cast<unsigned char*>(g_scratch_dev[dev]);
    return cudaSuccess;
}

struct Carver {
    unsigned char* base;
    size_t used = 0;
    bool ok = true;
    template <class T>
    T* take(size_t count) {
        size_t at = (used + 255) / 256 * 256;
        size_t bytes = sizeof(T) * std::max<size_t>(count, 1);
        if (at + bytes > kScratchBytes) { ok = false; return nullptr; }
        used = at + bytes;
        return reinterpret_cast<T*>(base + at);
    }
};

int bits_for_tiles(uint64_t n) {
    int b = 0;
    while (b < 63 && (1ull << b) < n) ++b;
    return b;
}

}  // namespace

extern "C" int dgs_render_noalloc(const dgs_options* opt, const dgs_node* nodes, int32_t n_nodes,
                                  const int32_t* env_node_ids, int32_t n_envs, int32_t max_nodes,
                                  const float* node_poses, const dgs_camera* cams, const int32_t* cams_per_env,
                                  int32_t max_cams, float* out_rgb, float* out_depth, float* out_alpha,
                                  const int64_t* view_pixel_offset, void* stream_) {
    dgs_options o;
    if (opt) o = *opt; else dgs_default_options(&o);
    std::string why;
    if (!check_options(&o, why)) return DGS_ERR_INVALID_ARG;
    cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_);
    // ---------------------------------------------------------------- validation and host tables (as dgs_render)
    HostTables H;
    const int vrc = build_host_tables(o, nodes, n_nodes, env_node_ids, n_envs, max_nodes, node_poses, cams, cams_per_env,
                                      max_cams, view_pixel_offset, H, why);
    if (vrc != DGS_OK) return vrc;
    if (!out_rgb || !out_depth) return DGS_ERR_INVALID_ARG;
    const int K = max_nodes;
    const int V = (int)H.views.size();
    if (V == 0) return DGS_OK;
    const std::vector<NodeDesc>& nd = H.nodes;
    const std::vector<ViewDesc>& views = H.views;
    const std::vector<int32_t>& slot_node = H.slot_node;
    const std::vector<int64_t>& vnode_tab = H.vnode_tab;
    const std::vector<int64_t>& view_tab = H.view_tab;
    const std::vector<int32_t>& nv_off = H.nv_off;
    const std::vector<NodeView>& nv = H.nv;
    const int dtype_mask = H.dtype_mask;
    const int64_t chunk_total = H.chunk_total, tiles_total = H.tiles_total, T = H.T;

    // ---------------------------------------------------------------- phase 1 scratch
    unsigned char* base = nullptr;
    if (scratch_address(&base) != cudaSuccess) return DGS_ERR_CUDA;
    Carver cv{base};
    NodeDesc* d_nodes = cv.take<NodeDesc>(n_nodes);
    ViewDesc* d_views = cv.take<ViewDesc>(V);
    int32_t* d_slot = cv.take<int32_t>((size_t)V * K);
    int64_t* d_vtab = cv.take<int64_t>((size_t)V * K);
    NodeView* d_nv = cv.take<NodeView>(nv.size());
    int32_t* d_nvoff = cv.take<int32_t>(n_nodes + 1);
    int64_t* d_viewtab = cv.take<int64_t>(V + 1);
    VNode* d_vnodes = cv.take<VNode>((size_t)V * K);
    uint32_t* d_err = cv.take<uint32_t>(kErrBlockBytes / 4);
    uint2* d_counts = cv.take<uint2>(T);
    uint32_t* d_inst_off = cv.take<uint32_t>(T + 1);
    uint64_t* d_pair_off = cv.take<uint64_t>(T + 1);
    const int64_t n_parts = (T + 4095) / 4096;
    ulonglong2* d_parts = cv.take<ulonglong2>(n_parts + 1);
    uint64_t* d_rb = cv.take<uint64_t>(2 * (V + 1) + 1);
    if (!cv.ok) return DGS_ERR_CAPACITY;

#define NA_CUDA(x) do { if ((x) != cudaSuccess) return DGS_ERR_CUDA; } while (0)
    // pageable copies: the runtime stages them, nothing is allocated here
    NA_CUDA(cudaMemcpyAsync(d_nodes, nd.data(), sizeof(NodeDesc) * n_nodes, cudaMemcpyHostToDevice, stream));
    NA_CUDA(cudaMemcpyAsync(d_views, views.data(), sizeof(ViewDesc) * V, cudaMemcpyHostToDevice, stream));
    NA_CUDA(cudaMemcpyAsync(d_slot, slot_node.data(), sizeof(int32_t) * V * K, cudaMemcpyHostToDevice, stream));
    NA_CUDA(cudaMemcpyAsync(d_vtab, vnode_tab.data(), sizeof(int64_t) * V * K, cudaMemcpyHostToDevice, stream));
    if (!nv.empty()) NA_CUDA(cudaMemcpyAsync(d_nv, nv.data(), sizeof(NodeView) * nv.size(), cudaMemcpyHostToDevice, stream));
    NA_CUDA(cudaMemcpyAsync(d_nvoff, nv_off.data(), sizeof(int32_t) * (n_nodes + 1), cudaMemcpyHostToDevice, stream));
    NA_CUDA(cudaMemcpyAsync(d_viewtab, view_tab.data(), sizeof(int64_t) * (V + 1), cudaMemcpyHostToDevice, stream));
    NA_CUDA(cudaMemsetAsync(d_err, 0, kErrBlockBytes, stream));

    Params P = make_params(o);
    P.err = d_err;
    int64_t launches = 0;
    Launch L{stream, &launches};
    launch_setup_views(L, d_views, V, node_poses, d_slot, K, d_vnodes, d_vtab, d_err);
    launch_count(L, dtype_mask, d_nodes, n_nodes, d_views, d_vnodes, K, d_nv, d_nvoff, (int)chunk_total, P, 0, V, true,
                 nullptr, 0, d_counts);
    launch_scan(L, d_counts, T, d_inst_off, d_pair_off, d_parts, n_parts + 1);
    // one view group: read back the grand totals and the error word
    NA_CUDA(cudaMemsetAsync(d_rb, 0, sizeof(uint64_t) * 3, stream));
    // the 64-bit instance total of the scan (its 32-bit offsets wrap beyond 2^32)
    if (n_parts > 0)
        NA_CUDA(cudaMemcpyAsync(d_rb, d_parts + n_parts, sizeof(uint64_t), cudaMemcpyDeviceToDevice, stream));
    NA_CUDA(cudaMemcpyAsync(d_rb + 1, d_pair_off + T, sizeof(uint64_t), cudaMemcpyDeviceToDevice, stream));
    NA_CUDA(cudaMemcpyAsync(d_rb + 2, d_err, sizeof(uint32_t), cudaMemcpyDeviceToDevice, stream));
    uint64_t h_rb[3] = {0, 0, 0};
    NA_CUDA(cudaMemcpyAsync(h_rb, d_rb, sizeof(uint64_t) * 3, cudaMemcpyDeviceToHost, stream));
    NA_CUDA(cudaGetLastError());
    NA_CUDA(cudaStreamSynchronize(stream));
    const uint64_t n_vis = h_rb[0], n_pairs = h_rb[1];
    if ((uint32_t)h_rb[2] & kErrPose) return DGS_ERR_INVALID_ARG;
    if (n_pairs > kMaxPairs || n_vis >= (1ull << 32)) return DGS_ERR_CAPACITY;

    // ---------------------------------------------------------------- phase 2 scratch
    const uint64_t ni = std::max<uint64_t>(n_vis, 1), np = std::max<uint64_t>(n_pairs, 1);
    Record* d_rec = cv.take<Record>(ni);
    InstInfo* d_info = cv.take<InstInfo>(ni);
    uint32_t* d_dk0 = cv.take<uint32_t>(ni);
    uint32_t* d_iv0 = cv.take<uint32_t>(ni);
    uint32_t* d_dk1 = cv.take<uint32_t>(ni);
    uint32_t* d_iv1 = cv.take<uint32_t>(ni);
    uint32_t* d_ntile = cv.take<uint32_t>(ni);
    uint32_t* d_vig = cv.take<uint32_t>(ni);
    uint32_t* d_poff = cv.take<uint32_t>(ni + 1);
    uint32_t* d_tparts = cv.take<uint32_t>(tile_scan_parts((uint32_t)ni));
    uint32_t* d_k0 = cv.take<uint32_t>(np);
    uint32_t* d_v0 = cv.take<uint32_t>(np);
    uint32_t* d_k1 = cv.take<uint32_t>(np);
    uint32_t* d_v1 = cv.take<uint32_t>(np);
    uint32_t* d_hist = cv.take<uint32_t>(8 * 256);
    uint32_t* d_cnt = cv.take<uint32_t>(8);
    uint32_t* d_total = cv.take<uint32_t>(1);
    uint32_t* d_status = cv.take<uint32_t>(sort_status_words((uint32_t)std::max(ni, np)));
    uint2* d_ranges = cv.take<uint2>((size_t)tiles_total);
    if (!cv.ok) return DGS_ERR_CAPACITY;
    // tile keys: view << tbits | tile in view, as in dgs_render with one view group
    int64_t max_view_tiles = 1;
    for (const ViewDesc& vd : views) max_view_tiles = std::max<int64_t>(max_view_tiles, (int64_t)vd.tiles_x * vd.tiles_y);
    const int tbits = bits_for_tiles((uint64_t)max_view_tiles + 1);
    if (tbits > kTileBits || tiles_total > kMaxGroupTiles || (int64_t)V >= (1ll << (kTileBits - tbits)))
        return DGS_ERR_CAPACITY;
    // depth-ordered tile lists, as in dgs_render with one view group
    // the depth sort's view key, packed into the instance numbers where both fit in 32 bits
    ViewKey vk;
    vk.bits = bits_for_tiles((uint64_t)V);
    if (vk.bits > 0 && bits_for_tiles(n_vis) + vk.bits <= 32) vk.vshift = 32 - vk.bits;
    vk.vig = vk.bits > 0 && !vk.vshift ? d_vig : nullptr;
    vk.inst_off = d_inst_off;
    vk.view_tab = d_viewtab;
    vk.v0 = 0;
    vk.nv = V;
    P.n_rec = (uint32_t)n_vis;
    P.view0 = 0;
    P.tbits = tbits;
    P.vshift = vk.vshift;
    launch_emit(L, dtype_mask, d_nodes, n_nodes, d_views, d_vnodes, K, d_nv, d_nvoff, (int)chunk_total, P, 0, V, true,
                nullptr, 0, d_counts, d_inst_off, 0u, d_rec, d_info, d_dk0, d_iv0, d_ntile, vk.vig ? d_vig : nullptr);
    uint32_t *dk, *order, *tk, *tv;
    SortCtl depth_ctl;
    depth_ctl.runs = true;
    launch_sort(L, d_dk0, d_iv0, d_dk1, d_iv1, (uint32_t)n_vis, kZBits, d_hist, d_status, d_cnt, d_err, &dk, &order,
                nullptr, depth_ctl, &vk);
    launch_tile_scan(L, order, d_ntile, (uint32_t)n_vis, nullptr, d_poff, d_tparts, (uint32_t)n_pairs, d_total, d_err);
    launch_pairs(L, d_views, K, order, d_poff, d_rec, d_info, (uint32_t)n_vis, nullptr, P, d_k0, d_v0, (uint32_t)n_pairs);
    SortCtl tile_ctl;
    tile_ctl.runs = true;
    launch_sort(L, d_k0, d_v0, d_k1, d_v1, (uint32_t)n_pairs, tbits, d_hist, d_status, d_cnt, d_err, &tk, &tv, d_total,
                tile_ctl);
    launch_ranges(L, tk, (uint32_t)n_pairs, d_ranges, (int)tiles_total, d_total, d_views, V, P);
    launch_composite(L, d_views, 0, V, (int)tiles_total, d_ranges, tk, tv, d_rec, P, out_rgb, out_depth, out_alpha,
                     nullptr);
    uint32_t h_err = 0;
    NA_CUDA(cudaMemcpyAsync(&h_err, d_err, sizeof(uint32_t), cudaMemcpyDeviceToHost, stream));
    NA_CUDA(cudaGetLastError());
    NA_CUDA(cudaStreamSynchronize(stream));
    if (h_err & kErrTimeout) return DGS_ERR_TIMEOUT;
    if (h_err & (kErrMismatch | kErrCapacity | kErrBounds)) return DGS_ERR_CUDA;
    if (h_err & kErrPose) return DGS_ERR_INVALID_ARG;
    return DGS_OK;
#undef NA_CUDA
}
