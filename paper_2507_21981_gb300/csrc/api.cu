// libdgs C ABI: contexts, argument validation, workspace and the render sequence.
//
// A call renders every (env, camera) view of a batch (Sec. III-C: RGB and depth sensors of
// many parallel environments, Sec. III-B: background + posed interactive nodes):
//   setup     camera_from_node per (view, slot), pose validation            (K0)
//   count     per (view, 32-Gaussian chunk): mask of visible lanes, tile pairs (K1)
//   scan      exclusive offsets of that table; per-view totals read back once
//   per view group: emit records + pairs (K2), radix sort (K3), tile ranges (K4),
//                   composite RGB + depth (K5)
// Plain mode makes every view its own group and launches its count/emit per view; batched
// mode counts all views in one launch (each Gaussian's attributes read once) and emits,
// sorts and composites as few groups as the 2^30-pair limit of the sort allows.
// dgs_render_backward rebuilds the same lists and runs the adjoint kernels instead of K5.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <memory>
#include <string>
#include <vector>

#include "dgs_internal.cuh"

using namespace dgs;

namespace {

struct DevBuf {
    void* p = nullptr;
    size_t bytes = 0;
};

struct TimedRange {
    int cls;
    cudaEvent_t a, b;
};

}  // namespace

// What a captured launch sequence depends on: every size that shapes a grid or a table
// layout, and every pointer baked into a kernel argument (workspace pointers through `gen`).
struct GraphKey {
    int64_t V, K, n_nodes, dtype_mask, chunk_total, T, tiles_total, n_nv, upload_bytes, meta_bytes;
    const void *poses, *rgb, *depth, *alpha;
    uint64_t gen;
    int64_t tile_w, tile_h, exact_tile_test;
    int64_t ng, split;
    const void* overlay;
    int64_t aug_on, ov_n, ov_w, ov_h;
};

// Workspace of one view group's lists.  dkey/ival: depth keys and instance numbers (depth
// sort, ping-pong); ntile: pairs per instance; poff/tparts: pair offsets in depth order;
// tkeys/tvals: (tile, instance) pairs (tile sort, ping-pong); ranges: per tile.
struct ListBufs {
    DevBuf records, info, dkey0, ival0, dkey1, ival1, ntile, poff, tparts, tkeys0, tvals0, tkeys1, tvals1, hist,
        status, counters, ranges, torder, ck_st, ck_off, ck_last, ck_jobs, ck_njobs, vig;
    static constexpr int kCount = 24;
    DevBuf* all[kCount] = {&records, &info, &dkey0, &ival0, &dkey1, &ival1, &ntile, &poff, &tparts, &tkeys0, &tvals0,
                           &tkeys1, &tvals1, &hist, &status, &counters, &ranges, &torder, &ck_st, &ck_off, &ck_last,
                           &ck_jobs, &ck_njobs, &vig};
    ListBufs() = default;
    ListBufs(const ListBufs&) = delete;
    ListBufs& operator=(const ListBufs&) = delete;
};

namespace {
struct SavedForward;   // an eager render's lists kept for its backward (dgs_options.keep_lists)
}  // namespace

struct dgs_ctx {
    dgs_options opt{};
    std::unique_ptr<SavedForward> saved;  // valid until the next call stages a batch
    std::string err;
    int device = 0;
    DevBuf meta, counts, inst_off, pair_off, parts, errword, readback, inst_grad, gsizes, totals;
    ListBufs lists[2];                    // view groups alternate between two sets (two streams)
    cudaStream_t aux_stream = nullptr;    // second stream of the eager sequence
    uint64_t gen = 0;                     // bumped whenever a workspace buffer is reallocated
    // graph replay (DGS_MODE_GRAPH)
    cudaStream_t cap_stream = nullptr;    // capture stream (the caller's may be the legacy stream)
    cudaStream_t cap_stream2 = nullptr;   // second capture stream (the second view group)
    cudaGraphExec_t gexec = nullptr;
    GraphKey gkey{};
    int gng = 1, gsplit = 0;              // captured view groups: [0, gsplit) and [gsplit, V)
    uint64_t cap_inst[2] = {0, 0}, cap_pairs[2] = {0, 0};  // capacities of each captured group
    int gbits = 0;
    int64_t glaunches = 0;
    // per captured group: its views, tiles, final sort buffers and parameters (keep_lists)
    int gv0[2] = {0, 0}, gv1[2] = {0, 0}, gtiles[2] = {0, 0};
    const uint32_t* gkeys[2] = {nullptr, nullptr};
    const uint32_t* gvals[2] = {nullptr, nullptr};
    const uint32_t* gorder[2] = {nullptr, nullptr};
    Params gP[2]{};
    Checkpoints gck[2]{};
    uint32_t gjobs[2] = {0, 0};
    int32_t captures = 0;
    void* h_graph = nullptr;              // pinned: error word + live totals after a replay
    void* h_meta = nullptr;
    size_t h_meta_bytes = 0;
    void* h_read = nullptr;
    size_t h_read_bytes = 0;
    dgs_stats stats{};
    float ktimes[DGS_K_COUNT_CLASSES] = {};
    int64_t launches = 0;
    std::vector<cudaEvent_t> events;
    std::vector<TimedRange> ranges_timed;
    size_t next_event = 0;
    // image randomisation (dgs_set_augment): per-view records, overlay clip
    std::vector<dgs_augment> aug;
    const uint8_t* overlay = nullptr;
    int32_t ov_n = 0, ov_w = 0, ov_h = 0;
    DevBuf aug_dev;                       // dgs_augment_rgb: spans + records
    void* h_aug = nullptr;                // its pinned staging
    size_t h_aug_bytes = 0;
    cudaEvent_t aug_copied = nullptr;     // the staging's last upload has been read
    // TSDF fusion: view table (device), its pinned staging and the event guarding the staging
    DevBuf tsdf_meta, tsdf_depth;
    void* h_tsdf = nullptr;
    size_t h_tsdf_bytes = 0;
    cudaEvent_t tsdf_copied = nullptr;
    // LiDAR (dgs_lidar_build / dgs_lidar_trace)
    DevBuf lid_rec, lid_box, lid_tab, lid_meta, lid_slots;
    std::vector<dgs_node> lid_nodes;      // the nodes the structures were built from
    void* h_lid = nullptr;                // pinned staging of the per-call tables
    size_t h_lid_bytes = 0;
};

namespace {

int fail(dgs_ctx* ctx, int code, const std::string& msg) {
    if (ctx) ctx->err = msg;
    return code;
}

const char* dbg_site_name(uint32_t site) {
    static const char* const names[kSiteCount] = {
        "unknown site", "emission: record number of a visible instance",
        "tile-count scan: depth-sorted instance number", "pair writer: depth-sorted instance number",
        "radix sort: destination of a live key", "compositor: instance number of a tile-list entry",
        "adjoint compositor: instance number of a tile-list entry",
        "projection adjoint: Gaussian of an instance within its node"};
    return site < kSiteCount ? names[site] : names[0];
}

std::string bounds_message(const uint32_t* block) {
    uint64_t idx = 0, bound = 0;
    std::memcpy(&idx, block + 2, sizeof(idx));
    std::memcpy(&bound, block + 4, sizeof(bound));
    return std::string("debug bounds check failed (") + dbg_site_name(block[0]) + "): index " + std::to_string(idx) +
           ", bound " + std::to_string(bound);
}

// A failed debug bounds check (kErrBounds): reads the block's record of it back.
int bounds_failure(dgs_ctx* ctx, const uint32_t* d_err) {
    uint32_t block[6] = {};
    cudaDeviceSynchronize();
    if (cudaMemcpy(block, d_err + kDbgWord, sizeof(block), cudaMemcpyDeviceToHost) != cudaSuccess)
        return fail(ctx, DGS_ERR_CUDA, "debug bounds check failed (site not readable)");
    return fail(ctx, DGS_ERR_CUDA, bounds_message(block));
}

int cuda_fail(dgs_ctx* ctx, cudaError_t e, const char* what) {
    return fail(ctx, e == cudaErrorMemoryAllocation ? DGS_ERR_OOM : DGS_ERR_CUDA,
                std::string(what) + ": " + cudaGetErrorString(e));
}

#define DGS_CUDA(ctx, call)                                        \
    do {                                                           \
        cudaError_t e_ = (call);                                   \
        if (e_ != cudaSuccess) return cuda_fail(ctx, e_, #call);   \
    } while (0)

int ensure(dgs_ctx* ctx, DevBuf& b, size_t bytes) {
    if (bytes <= b.bytes) return DGS_OK;
    if (b.p) {
        cudaError_t e = cudaFree(b.p);
        b.p = nullptr;
        b.bytes = 0;
        if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaFree");
    }
    ++ctx->gen;
    size_t want = std::max<size_t>(bytes + bytes / 4, 256);
    cudaError_t e = cudaMalloc(&b.p, want);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return cuda_fail(ctx, e, "cudaMalloc");
    }
    b.bytes = want;
    return DGS_OK;
}

int ensure_host(dgs_ctx* ctx, void*& p, size_t& have, size_t bytes) {
    if (bytes <= have) return DGS_OK;
    if (p) cudaFreeHost(p);
    p = nullptr;
    have = 0;
    size_t want = std::max<size_t>(bytes + bytes / 4, 4096);
    cudaError_t e = cudaMallocHost(&p, want);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaMallocHost");
    have = want;
    return DGS_OK;
}

void free_buf(DevBuf& b) {
    if (b.p) cudaFree(b.p);
    b.p = nullptr;
    b.bytes = 0;
}

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

bool finite(float x) { return std::isfinite(x); }

cudaEvent_t take_event(dgs_ctx* ctx) {
    if (ctx->next_event == ctx->events.size()) {
        cudaEvent_t e;
        cudaEventCreate(&e);
        ctx->events.push_back(e);
    }
    return ctx->events[ctx->next_event++];
}

struct Timer {
    dgs_ctx* ctx;
    cudaStream_t s;
    bool on;
    cudaEvent_t a{};

    int cls = -1;
    void begin(int c) {
        if (!on) return;
        cls = c;
        a = take_event(ctx);
        cudaEventRecord(a, s);
    }
    void end() {
        if (!on || cls < 0) return;
        cudaEvent_t b = take_event(ctx);
        cudaEventRecord(b, s);
        ctx->ranges_timed.push_back({cls, a, b});
        cls = -1;
    }
};

// After the stream has been synchronised: the profiled ranges' times into ctx->ktimes.
void collect_times(dgs_ctx* ctx) {
    if (!ctx->opt.profile) return;
    for (const TimedRange& r : ctx->ranges_timed) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) ctx->ktimes[r.cls] += ms;
    }
}

// Per-view exclusive offsets of instances and pairs into out[0, n) and out[n, 2n); out[2n + 1]
// receives the 64-bit instance total of the count scan (the 32-bit offsets wrap beyond 2^32).
__global__ void k_view_totals(const uint32_t* __restrict__ inst_off, const uint64_t* __restrict__ pair_off,
                              const int64_t* __restrict__ view_tab, int n, const ulonglong2* __restrict__ scan_total,
                              uint64_t* out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    out[i] = inst_off[view_tab[i]];
    out[n + i] = pair_off[view_tab[i]];
    if (i == 0) out[2 * n + 1] = scan_total ? scan_total->x : 0ull;
}

constexpr uint64_t kPipelinePairs = 1ull << 22;   // batches with this many pairs run as two groups

int bits_for(uint64_t n) {   // smallest b with 2^b >= n (n >= 1)
    int b = 0;
    while (b < 63 && (1ull << b) < n) ++b;
    return b;
}

}  // namespace

namespace dgs {

int check_options(const dgs_options* o, std::string& why) {
    if (o->mode != DGS_MODE_PLAIN && o->mode != DGS_MODE_BATCHED && o->mode != DGS_MODE_GRAPH) {
        why = "mode";
        return 0;
    }
    const int area = o->tile_w * o->tile_h;
    // w = 8a, h = 4b with 32ab in {64, 128, 256}: both are powers of two
    if (o->tile_w < 8 || o->tile_h < 4 || o->tile_w % 8 || o->tile_h % 4 || (area != 64 && area != 128 && area != 256) ||
        (o->tile_w & (o->tile_w - 1)) || (o->tile_h & (o->tile_h - 1))) {
        why = "tile shape";
        return 0;
    }
    if (!(o->z_near > 0) || !finite(o->z_near)) { why = "z_near"; return 0; }
    if (!(o->lowpass >= 0) || !finite(o->lowpass)) { why = "lowpass"; return 0; }
    if (!(o->alpha_min >= 0) || !(o->alpha_max > 0) || !(o->alpha_max <= 1)) { why = "alpha limits"; return 0; }
    if (!(o->t_min >= 0) || !(o->t_min < 1)) { why = "t_min"; return 0; }
    if (!(o->q_max > 0) || !finite(o->q_max)) { why = "q_max"; return 0; }
    if (!(o->guard > 0) || !finite(o->guard)) { why = "guard"; return 0; }
    for (int i = 0; i < 3; ++i) if (!finite(o->bg[i])) { why = "bg"; return 0; }
    if (o->views_per_group < 0) { why = "views_per_group"; return 0; }
    if (o->spin_limit_us < 0) { why = "spin_limit_us"; return 0; }
    if (o->check_binning < 0 || o->check_binning > 1) { why = "check_binning"; return 0; }
    if (o->test_fault < 0 || o->test_fault > 4) { why = "test_fault"; return 0; }
    if (o->test_fault == 3 && !kDebugChecks) { why = "test_fault 3 (needs a DGS_DEBUG build)"; return 0; }
    if (o->keep_lists < 0 || o->keep_lists > 1) { why = "keep_lists"; return 0; }
    return 1;
}

Params make_params(const dgs_options& o) {
    Params P{};
    P.z_near = o.z_near; P.lowpass = o.lowpass; P.alpha_min = o.alpha_min; P.alpha_max = o.alpha_max;
    P.t_min = o.t_min; P.q_max = o.q_max; P.guard = o.guard;
    P.bg0 = o.bg[0]; P.bg1 = o.bg[1]; P.bg2 = o.bg[2];
    P.qbin = o.q_max * 1.001f + 1e-3f;
    P.p_min = kHalfLog2e * o.q_max;
    P.log2_amin = o.alpha_min > 0.f ? std::log2(o.alpha_min) : -INFINITY;
    P.tile_w = o.tile_w; P.tile_h = o.tile_h;
    while ((1 << P.tile_sx) < o.tile_w) ++P.tile_sx;
    while ((1 << P.tile_sy) < o.tile_h) ++P.tile_sy;
    P.exact_tile_test = o.exact_tile_test;
    uint32_t b;
    std::memcpy(&b, &o.z_near, 4);
    P.zbase = b & 0x7F800000u;   // 2^floor(log2 z_near)
    return P;
}

// Argument validation and the host tables of one batch (see HostTables).  Returns DGS_OK, or
// the status of the first failed check with its description in `why`.  No CUDA call.
int build_host_tables(const dgs_options& o, const dgs_node* nodes, int32_t n_nodes, const int32_t* env_node_ids,
                      int32_t n_envs, int32_t max_nodes, const float* node_poses, const dgs_camera* cams,
                      const int32_t* cams_per_env, int32_t max_cams, const int64_t* view_pixel_offset, HostTables& H,
                      std::string& why) {
    auto reject = [](std::string& w, int code, const std::string& msg) { w = msg; return code; };
    // ---------------------------------------------------------------- validation (synchronous)
    if (n_nodes < 1 || !nodes) return reject(why, DGS_ERR_INVALID_ARG, "nodes: need n_nodes >= 1 and a node array");
    if (n_envs < 1 || max_nodes < 1 || max_cams < 1) return reject(why, DGS_ERR_INVALID_ARG, "n_envs, max_nodes, max_cams must be >= 1");
    if (!env_node_ids || !cams || !cams_per_env || !node_poses) return reject(why, DGS_ERR_INVALID_ARG, "null table pointer");
    int64_t total_gauss = 0;
    for (int k = 0; k < n_nodes; ++k) {
        const dgs_node& nd = nodes[k];
        if (nd.n < 0 || nd.sh_degree < 0 || nd.sh_degree > 3 || nd.dtype < 0 || nd.dtype > 2)
            return reject(why, DGS_ERR_INVALID_ARG, "node " + std::to_string(k) + ": bad n, sh_degree or dtype");
        if (nd.n > 0 && (!nd.mean || !nd.log_scale || !nd.quat || !nd.opacity_logit || !nd.sh))
            return reject(why, DGS_ERR_INVALID_ARG, "node " + std::to_string(k) + ": null attribute pointer");
        total_gauss += nd.n;
    }
    if (total_gauss >= (1ll << 32)) return reject(why, DGS_ERR_INVALID_ARG, "more than 2^32 Gaussians");
    const int E = n_envs, K = max_nodes, C = max_cams;
    std::vector<int> seen(n_nodes, -1);
    for (int e = 0; e < E; ++e) {
        for (int j = 0; j < K; ++j) {
            const int k = env_node_ids[(int64_t)e * K + j];
            if (k < -1 || k >= n_nodes) return reject(why, DGS_ERR_INVALID_ARG, "env_node_ids out of range");
            if (k >= 0) {
                if (seen[k] == e) return reject(why, DGS_ERR_INVALID_ARG, "a node appears twice in one env");
                seen[k] = e;
            }
        }
        if (cams_per_env[e] < 0 || cams_per_env[e] > C) return reject(why, DGS_ERR_INVALID_ARG, "cams_per_env out of range");
    }
    // views
    std::vector<ViewDesc> views;
    std::vector<int> view_env, view_cam;
    int64_t tiles_total = 0, pix_total = 0;
    for (int e = 0; e < E; ++e)
        for (int c = 0; c < cams_per_env[e]; ++c) {
            const dgs_camera& cm = cams[(int64_t)e * C + c];
            if (cm.width < 1 || cm.height < 1 || cm.width > 32768 || cm.height > 32768)
                return reject(why, DGS_ERR_INVALID_ARG, "camera resolution");
            if (!(cm.fx > 0) || !(cm.fy > 0) || !finite(cm.fx) || !finite(cm.fy) || !finite(cm.cx) || !finite(cm.cy))
                return reject(why, DGS_ERR_INVALID_ARG, "camera intrinsics");
            for (int a = 0; a < 12; ++a)
                if (!finite(cm.cam_from_world[a])) return reject(why, DGS_ERR_INVALID_ARG, "camera pose not finite");
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b) {
                    double s = 0;
                    for (int r = 0; r < 3; ++r) s += (double)cm.cam_from_world[r * 4 + a] * cm.cam_from_world[r * 4 + b];
                    if (std::fabs(s - (a == b ? 1.0 : 0.0)) > 1e-4) return reject(why, DGS_ERR_INVALID_ARG, "camera rotation not orthonormal");
                }
            ViewDesc vd{};
            vd.fx = cm.fx; vd.fy = cm.fy; vd.cx = cm.cx; vd.cy = cm.cy;
            vd.limx = o.guard * 0.5f * (float)cm.width / cm.fx;
            vd.limy = o.guard * 0.5f * (float)cm.height / cm.fy;
            vd.W = cm.width; vd.H = cm.height;
            vd.tiles_x = (cm.width + o.tile_w - 1) / o.tile_w;
            vd.tiles_y = (cm.height + o.tile_h - 1) / o.tile_h;
            vd.env = e;
            vd.tile_base = (int32_t)tiles_total;
            std::memcpy(vd.cam, cm.cam_from_world, sizeof(vd.cam));
            tiles_total += (int64_t)vd.tiles_x * vd.tiles_y;
            if (tiles_total >= (1ll << 31)) return reject(why, DGS_ERR_INVALID_ARG, "too many tiles");
            const int64_t v = (int64_t)views.size();
            vd.pix_off = view_pixel_offset ? view_pixel_offset[v] : pix_total;
            if (vd.pix_off < 0) return reject(why, DGS_ERR_INVALID_ARG, "negative view_pixel_offset");
            pix_total += (int64_t)cm.width * cm.height;
            views.push_back(vd);
            view_env.push_back(e);
            view_cam.push_back(c);
        }
    const int V = (int)views.size();
    H.pix_total = pix_total;
    if (V == 0) {
        H.views = std::move(views);
        return DGS_OK;
    }

    // ---------------------------------------------------------------- host tables
    std::vector<NodeDesc> nd(n_nodes);
    int dtype_mask = 0;
    int64_t chunk_total = 0, gbase = 0;
    for (int k = 0; k < n_nodes; ++k) {
        nd[k].mean = nodes[k].mean; nd[k].log_scale = nodes[k].log_scale; nd[k].quat = nodes[k].quat;
        nd[k].opac = nodes[k].opacity_logit; nd[k].sh = nodes[k].sh;
        nd[k].n = nodes[k].n; nd[k].gbase = gbase; nd[k].deg = nodes[k].sh_degree; nd[k].dtype = nodes[k].dtype;
        nd[k].chunk0 = (int32_t)chunk_total;
        nd[k].nchunks = (int32_t)((nodes[k].n + kChunk - 1) / kChunk);
        chunk_total += nd[k].nchunks;
        gbase += nodes[k].n;
        if (nodes[k].n > 0) dtype_mask |= 1 << nodes[k].dtype;
    }
    if (chunk_total >= (1ll << 31)) return reject(why, DGS_ERR_INVALID_ARG, "too many Gaussians");
    // count table: per view, the chunks of its nodes in node-id order
    std::vector<int32_t> slot_node((size_t)V * K, -1);
    std::vector<int64_t> vnode_tab((size_t)V * K, 0), view_tab(V + 1, 0);
    std::vector<int32_t> pmap((size_t)V * (2 * K + 1), 0);
    std::vector<std::vector<NodeView>> per_node(n_nodes);
    int64_t tab = 0, n_instances = 0;
    for (int v = 0; v < V; ++v) {
        const int e = view_env[v];
        std::vector<std::pair<int, int>> present;   // (node, slot)
        for (int j = 0; j < K; ++j) {
            const int k = env_node_ids[(int64_t)e * K + j];
            slot_node[(size_t)v * K + j] = k;
            if (k >= 0) present.push_back({k, j});
        }
        std::sort(present.begin(), present.end());
        view_tab[v] = tab;
        int32_t* pm = &pmap[(size_t)v * (2 * K + 1)];
        int32_t pre = 0;
        for (size_t i = 0; i < present.size(); ++i) {
            const int k = present[i].first, j = present[i].second;
            vnode_tab[(size_t)v * K + j] = tab;
            pm[i] = pre;
            pm[K + 1 + i] = j;
            pre += nd[k].nchunks;
            tab += nd[k].nchunks;
            n_instances += nd[k].n;
            per_node[k].push_back({v, j, vnode_tab[(size_t)v * K + j]});
        }
        for (int i = (int)present.size(); i <= K; ++i) pm[i] = pre;
        for (int i = (int)present.size(); i < K; ++i) pm[K + 1 + i] = present.empty() ? 0 : present[0].second;
    }
    view_tab[V] = tab;
    const int64_t T = tab;
    std::vector<int32_t> nv_off(n_nodes + 1, 0);
    std::vector<NodeView> nv;
    for (int k = 0; k < n_nodes; ++k) {
        nv_off[k] = (int32_t)nv.size();
        nv.insert(nv.end(), per_node[k].begin(), per_node[k].end());
    }
    nv_off[n_nodes] = (int32_t)nv.size();
    H.nodes = std::move(nd);
    H.views = std::move(views);
    H.view_env = std::move(view_env);
    H.view_cam = std::move(view_cam);
    H.slot_node = std::move(slot_node);
    H.vnode_tab = std::move(vnode_tab);
    H.view_tab = std::move(view_tab);
    H.pmap = std::move(pmap);
    H.nv_off = std::move(nv_off);
    H.nv = std::move(nv);
    H.dtype_mask = dtype_mask;
    H.chunk_total = chunk_total;
    H.tiles_total = tiles_total;
    H.n_instances = n_instances;
    H.T = T;
    return DGS_OK;
}


}  // namespace dgs

namespace {

// Everything one call needs after validation and the count pass.
struct Batch {
    int V = 0, K = 0, n_nodes = 0;
    int dtype_mask = 0;
    int64_t chunk_total = 0, tiles_total = 0, T = 0;
    bool batched = true;
    std::vector<ViewDesc> views;
    std::vector<int64_t> view_tab;
    std::vector<std::pair<int, int>> groups;
    const uint64_t* inst_at = nullptr;     // per-view exclusive instance offsets (host, V+1)
    const uint64_t* pair_at = nullptr;     // per-view exclusive pair offsets (host, V+1)
    const NodeDesc* d_nodes = nullptr;
    const ViewDesc* d_views = nullptr;
    const NodeView* d_nv = nullptr;
    const int32_t* d_nvoff = nullptr;
    const int32_t* d_pmap = nullptr;
    VNode* d_vnodes = nullptr;
    uint2* d_counts = nullptr;
    uint32_t* d_inst_off = nullptr;
    uint64_t* d_pair_off = nullptr;
    uint32_t* d_err = nullptr;
    const dgs_node_grads* d_grads = nullptr;
    const int32_t* d_slot = nullptr;
    const int64_t* d_vtab = nullptr;
    const int64_t* d_viewtab = nullptr;
    const float* node_poses = nullptr;
    int64_t n_parts = 0, n_nv = 0;
    size_t upload_bytes = 0, meta_bytes = 0;
    size_t front_bytes = 0;                // device bytes of the tables up to the count scan
    Params P{};
};

void invalidate_saved(dgs_ctx* ctx);

// Validation, host tables and their upload (one copy from pinned memory), workspace for the
// count table.  Returns DGS_OK with B filled (B.V == 0: nothing to render).
int stage(dgs_ctx* ctx, const dgs_node* nodes, int32_t n_nodes, const int32_t* env_node_ids, int32_t n_envs,
            int32_t max_nodes, const float* node_poses, const dgs_camera* cams, const int32_t* cams_per_env,
            int32_t max_cams, const float* out_rgb, const float* out_depth, const int64_t* view_pixel_offset,
            const dgs_node_grads* grads, cudaStream_t stream, Timer& tm, Batch& B, bool need_outputs = true) {
    const dgs_options& o = ctx->opt;
    invalidate_saved(ctx);   // the staging below overwrites the tables a kept forward refers to
    HostTables H;
    std::string why;
    const int vrc = build_host_tables(o, nodes, n_nodes, env_node_ids, n_envs, max_nodes, node_poses, cams, cams_per_env,
                                      max_cams, view_pixel_offset, H, why);
    if (vrc != DGS_OK) return fail(ctx, vrc, why);
    if (need_outputs && (!out_rgb || !out_depth)) return fail(ctx, DGS_ERR_INVALID_ARG, "out_rgb and out_depth are required");
    const int V = (int)H.views.size(), K = max_nodes;
    const bool aug_on = !ctx->aug.empty();
    if (aug_on && (int64_t)ctx->aug.size() != V)
        return fail(ctx, DGS_ERR_INVALID_ARG, "the randomisation is set for " + std::to_string(ctx->aug.size()) +
                                                  " views, the batch has " + std::to_string(V));
    ctx->stats = dgs_stats{};
    ctx->stats.n_views = V;
    ctx->stats.n_pixels = H.pix_total;
    for (float& t : ctx->ktimes) t = 0.f;
    B.V = V;
    if (V == 0) return DGS_OK;
    ctx->stats.n_instances = H.n_instances;
    std::vector<NodeDesc>& nd = H.nodes;
    std::vector<ViewDesc>& views = H.views;
    std::vector<int32_t>& slot_node = H.slot_node;
    std::vector<int64_t>& vnode_tab = H.vnode_tab;
    std::vector<int64_t>& view_tab = H.view_tab;
    std::vector<int32_t>& pmap = H.pmap;
    std::vector<int32_t>& nv_off = H.nv_off;
    std::vector<NodeView>& nv = H.nv;
    const int dtype_mask = H.dtype_mask;
    const int64_t chunk_total = H.chunk_total, tiles_total = H.tiles_total, T = H.T;

    // ---------------------------------------------------------------- upload (one copy)
    size_t off = 0;
    auto place = [&](size_t bytes) { size_t at = align_up(off, 256); off = at + bytes; return at; };
    const size_t o_nodes = place(sizeof(NodeDesc) * n_nodes);
    const size_t o_views = place(sizeof(ViewDesc) * V);
    const size_t o_slot = place(sizeof(int32_t) * V * K);
    const size_t o_vtab = place(sizeof(int64_t) * V * K);
    const size_t o_nv = place(sizeof(NodeView) * std::max<size_t>(1, nv.size()));
    const size_t o_nvoff = place(sizeof(int32_t) * (n_nodes + 1));
    const size_t o_pmap = place(sizeof(int32_t) * pmap.size());
    const size_t o_viewtab = place(sizeof(int64_t) * (V + 1));
    const size_t o_grads = place(sizeof(dgs_node_grads) * n_nodes);
    const size_t o_aug = aug_on ? place(sizeof(dgs_augment) * V) : 0;
    const size_t upload_bytes = off;
    const size_t o_vnodes = place(sizeof(VNode) * V * K);
    const size_t meta_bytes = off;
    int rc;
    if ((rc = ensure(ctx, ctx->meta, meta_bytes))) return rc;
    if ((rc = ensure_host(ctx, ctx->h_meta, ctx->h_meta_bytes, upload_bytes))) return rc;
    // the previous call's upload may still be in flight from this staging buffer
    DGS_CUDA(ctx, cudaStreamSynchronize(stream));
    char* hm = static_cast<char*>(ctx->h_meta);
    std::memcpy(hm + o_nodes, nd.data(), sizeof(NodeDesc) * n_nodes);
    std::memcpy(hm + o_views, views.data(), sizeof(ViewDesc) * V);
    std::memcpy(hm + o_slot, slot_node.data(), sizeof(int32_t) * V * K);
    std::memcpy(hm + o_vtab, vnode_tab.data(), sizeof(int64_t) * V * K);
    if (!nv.empty()) std::memcpy(hm + o_nv, nv.data(), sizeof(NodeView) * nv.size());
    std::memcpy(hm + o_nvoff, nv_off.data(), sizeof(int32_t) * (n_nodes + 1));
    std::memcpy(hm + o_pmap, pmap.data(), sizeof(int32_t) * pmap.size());
    std::memcpy(hm + o_viewtab, view_tab.data(), sizeof(int64_t) * (V + 1));
    if (grads) std::memcpy(hm + o_grads, grads, sizeof(dgs_node_grads) * n_nodes);
    else std::memset(hm + o_grads, 0, sizeof(dgs_node_grads) * n_nodes);
    if (aug_on) std::memcpy(hm + o_aug, ctx->aug.data(), sizeof(dgs_augment) * V);
    char* dm = static_cast<char*>(ctx->meta.p);
    const NodeDesc* d_nodes = reinterpret_cast<const NodeDesc*>(dm + o_nodes);
    const ViewDesc* d_views = reinterpret_cast<const ViewDesc*>(dm + o_views);
    const int32_t* d_slot = reinterpret_cast<const int32_t*>(dm + o_slot);
    const int64_t* d_vtab = reinterpret_cast<const int64_t*>(dm + o_vtab);
    const NodeView* d_nv = reinterpret_cast<const NodeView*>(dm + o_nv);
    const int32_t* d_nvoff = reinterpret_cast<const int32_t*>(dm + o_nvoff);
    const int32_t* d_pmap = reinterpret_cast<const int32_t*>(dm + o_pmap);
    const int64_t* d_viewtab = reinterpret_cast<const int64_t*>(dm + o_viewtab);
    VNode* d_vnodes = reinterpret_cast<VNode*>(dm + o_vnodes);

    if ((rc = ensure(ctx, ctx->errword, kErrBlockBytes))) return rc;
    if ((rc = ensure(ctx, ctx->counts, sizeof(uint2) * std::max<int64_t>(T, 1)))) return rc;
    if ((rc = ensure(ctx, ctx->inst_off, sizeof(uint32_t) * (T + 1)))) return rc;
    if ((rc = ensure(ctx, ctx->pair_off, sizeof(uint64_t) * (T + 1)))) return rc;
    const int64_t n_parts = (T + 4095) / 4096;
    if ((rc = ensure(ctx, ctx->parts, sizeof(ulonglong2) * (n_parts + 1)))) return rc;
    if ((rc = ensure(ctx, ctx->readback, sizeof(uint64_t) * 2 * (V + 1) + 64))) return rc;
    // pinned: per-view totals, the error word, then the exact pairs of every view group (<= V)
    if ((rc = ensure_host(ctx, ctx->h_read, ctx->h_read_bytes, sizeof(uint64_t) * 2 * (V + 1) + 64 + 4 * (V + 1))))
        return rc;
    if ((rc = ensure(ctx, ctx->totals, sizeof(uint32_t) * (V + 1)))) return rc;
    B.front_bytes = meta_bytes + 64 + sizeof(uint2) * std::max<int64_t>(T, 1) + sizeof(uint32_t) * (T + 1) +
                    sizeof(uint64_t) * (T + 1) + sizeof(ulonglong2) * (n_parts + 1) + sizeof(uint64_t) * 2 * (V + 1) +
                    64 + sizeof(uint32_t) * (V + 1);
    uint32_t* d_err = static_cast<uint32_t*>(ctx->errword.p);

    DGS_CUDA(ctx, cudaMemcpyAsync(dm, hm, upload_bytes, cudaMemcpyHostToDevice, stream));

    Params P = make_params(o);
    P.err = d_err;
    P.gate = nullptr;
    if (aug_on) {
        P.aug = reinterpret_cast<const dgs_augment*>(dm + o_aug);
        P.overlay = ctx->overlay;
        P.ov_w = ctx->ov_w;
        P.ov_h = ctx->ov_h;
    }
    B.K = K; B.n_nodes = n_nodes; B.dtype_mask = dtype_mask; B.chunk_total = chunk_total;
    B.tiles_total = tiles_total; B.T = T; B.batched = o.mode != DGS_MODE_PLAIN;
    // tile keys hold the view in the group above the tile's index in its view: its bits leave
    // the all-ones index (a dead pair's) above every real tile
    int64_t max_view_tiles = 1;
    for (const ViewDesc& vd : views) max_view_tiles = std::max<int64_t>(max_view_tiles, (int64_t)vd.tiles_x * vd.tiles_y);
    const int tbits = bits_for((uint64_t)max_view_tiles + 1);
    B.views = std::move(views); B.view_tab = std::move(view_tab);
    B.d_nodes = d_nodes; B.d_views = d_views; B.d_nv = d_nv; B.d_nvoff = d_nvoff; B.d_pmap = d_pmap;
    B.d_vnodes = d_vnodes; B.d_slot = d_slot; B.d_vtab = d_vtab; B.d_viewtab = d_viewtab;
    B.d_counts = static_cast<uint2*>(ctx->counts.p);
    B.d_inst_off = static_cast<uint32_t*>(ctx->inst_off.p);
    B.d_pair_off = static_cast<uint64_t*>(ctx->pair_off.p);
    B.d_err = d_err; B.P = P;
    B.P.tbits = tbits;
    B.d_grads = reinterpret_cast<const dgs_node_grads*>(dm + o_grads);
    B.node_poses = node_poses;
    B.n_parts = n_parts;
    B.n_nv = (int64_t)nv.size();
    B.upload_bytes = upload_bytes;
    B.meta_bytes = meta_bytes;
    return DGS_OK;
}

// Clears the error word, then setup (K0), count (K1) and the exclusive scan of the count table.
void launch_front(dgs_ctx* ctx, const Batch& B, const Launch& L, Timer& tm) {
    cudaMemsetAsync(B.d_err, 0, kErrBlockBytes, L.stream);
    tm.begin(DGS_K_SETUP);
    launch_setup_views(L, B.d_views, B.V, B.node_poses, B.d_slot, B.K, B.d_vnodes, B.d_vtab, B.d_err);
    tm.end();
    tm.begin(DGS_K_COUNT);
    if (B.batched) {
        launch_count(L, B.dtype_mask, B.d_nodes, B.n_nodes, B.d_views, B.d_vnodes, B.K, B.d_nv, B.d_nvoff,
                     (int)B.chunk_total, B.P, 0, B.V, true, nullptr, 0, B.d_counts);
    } else {
        for (int v = 0; v < B.V; ++v)
            launch_count(L, B.dtype_mask, B.d_nodes, B.n_nodes, B.d_views, B.d_vnodes, B.K, B.d_nv, B.d_nvoff,
                         (int)B.chunk_total, B.P, v, v + 1, false, B.d_pmap + (size_t)v * (2 * B.K + 1),
                         B.view_tab[v + 1] - B.view_tab[v], B.d_counts);
    }
    tm.end();
    tm.begin(DGS_K_SCAN);
    launch_scan(L, B.d_counts, B.T, B.d_inst_off, B.d_pair_off, static_cast<ulonglong2*>(ctx->parts.p), B.n_parts + 1);
    tm.end();
}

// Workspace of one set of group lists: n_inst instances, n_pairs tile pairs, n_tiles tiles.
// Bytes of each buffer of ListBufs (in ListBufs::all order) for one view group of n_inst
// instances, n_pairs tile pairs and n_tiles tiles.
// Compositor checkpoints of a group (keep_lists): slots for every segment after a tile's first,
// n_pairs / kSegEntries + 1 at most, of one CkState per pixel of each sub-tile; none beyond
// kMaxCheckpointBytes or kOrderMaxTiles tiles.
constexpr size_t kMaxCheckpointBytes = size_t(512) << 20;
uint64_t ck_slots(uint64_t n_pairs) { return n_pairs / kSegEntries + 1; }
size_t ck_state_bytes(uint64_t n_pairs, int64_t n_tiles, int tile_px) {
    if (n_tiles > kOrderMaxTiles) return 0;
    const size_t b = sizeof(CkState) * ck_slots(n_pairs) * (size_t)tile_px;
    return b <= kMaxCheckpointBytes ? b : 0;
}

void list_bytes(uint64_t n_inst, uint64_t n_pairs, int64_t n_tiles, int tile_px, bool with_ck,
                size_t out[ListBufs::kCount]) {
    n_inst = std::max<uint64_t>(n_inst, 1);
    n_pairs = std::max<uint64_t>(n_pairs, 1);
    const size_t u = sizeof(uint32_t);
    const size_t nt = (size_t)std::max<int64_t>(n_tiles, 1);
    const size_t ck = with_ck ? ck_state_bytes(n_pairs, n_tiles, tile_px) : 0;
    const size_t n_sub = (size_t)tile_px / 32;
    const size_t b[ListBufs::kCount] = {
        sizeof(Record) * n_inst, sizeof(InstInfo) * n_inst, u * n_inst, u * n_inst, u * n_inst,
        u * n_inst, u * n_inst, u * (n_inst + 1), u * tile_scan_parts((uint32_t)n_inst),
        u * n_pairs, u * n_pairs, u * n_pairs, u * n_pairs, u * 4 * 1024,
        u * sort_status_words((uint32_t)std::max(n_inst, n_pairs)), u * 8,
        sizeof(uint2) * nt, n_tiles <= kOrderMaxTiles ? u * nt : 0,
        ck, ck ? u * nt : 0, ck ? u * nt * n_sub : 0, ck ? sizeof(uint2) * (nt + ck_slots(n_pairs)) : 0, ck ? u : 0,
        u * n_inst};
    for (int i = 0; i < ListBufs::kCount; ++i) out[i] = b[i];
}

// Workspace of one set of group lists: n_inst instances, n_pairs tile pairs, n_tiles tiles.
int ensure_lists(dgs_ctx* ctx, ListBufs& lb, uint64_t n_inst, uint64_t n_pairs, int64_t n_tiles) {
    size_t bytes[ListBufs::kCount];
    list_bytes(n_inst, n_pairs, n_tiles, ctx->opt.tile_w * ctx->opt.tile_h, ctx->opt.keep_lists != 0, bytes);
    for (int i = 0; i < ListBufs::kCount; ++i) {
        const int rc = ensure(ctx, *lb.all[i], bytes[i]);
        if (rc) return rc;
    }
    return DGS_OK;
}

// Per-view totals read back once (one stream synchronisation), view groups and workspace
// sizing for the eager sequence.
int readback_groups(dgs_ctx* ctx, Batch& B, cudaStream_t stream, Timer& tm, size_t* need = nullptr) {
    const dgs_options& o = ctx->opt;
    const int V = B.V;
    int rc;
    tm.begin(DGS_K_SCAN);
    {
        uint64_t* d_rb = static_cast<uint64_t*>(ctx->readback.p);
        const ulonglong2* scan_total = B.n_parts > 0 ? static_cast<ulonglong2*>(ctx->parts.p) + B.n_parts : nullptr;
        k_view_totals<<<(V + 1 + 127) / 128, 128, 0, stream>>>(B.d_inst_off, B.d_pair_off, B.d_viewtab, V + 1,
                                                               scan_total, d_rb);
        ++ctx->launches;
        DGS_CUDA(ctx, cudaMemsetAsync(d_rb + 2 * (V + 1), 0, sizeof(uint64_t), stream));
        DGS_CUDA(ctx, cudaMemcpyAsync(d_rb + 2 * (V + 1), B.d_err, sizeof(uint32_t), cudaMemcpyDeviceToDevice, stream));
        DGS_CUDA(ctx, cudaMemcpyAsync(ctx->h_read, d_rb, sizeof(uint64_t) * 2 * (V + 1) + 16, cudaMemcpyDeviceToHost, stream));
    }
    tm.end();
    DGS_CUDA(ctx, cudaGetLastError());
    DGS_CUDA(ctx, cudaStreamSynchronize(stream));
    const uint64_t* h_rb = static_cast<const uint64_t*>(ctx->h_read);
    const uint64_t* inst_at = h_rb;
    const uint64_t* pair_at = h_rb + (V + 1);
    uint32_t errw = (uint32_t)(h_rb[2 * (V + 1)] & 0xFFFFFFFFu);
    if (errw & kErrPose) return fail(ctx, DGS_ERR_INVALID_ARG, "a node pose is not finite or not rigid");
    const uint64_t n_vis64 = h_rb[2 * (V + 1) + 1];
    ctx->stats.n_visible = (int64_t)n_vis64;
    if (n_vis64 >= (1ull << 32)) return fail(ctx, DGS_ERR_CAPACITY, "2^32 or more visible instances");

    // ---------------------------------------------------------------- groups
    std::vector<std::pair<int, int>> groups;
    if (!B.batched) {
        for (int v = 0; v < V; ++v) groups.push_back({v, v + 1});
    } else {
        int v0 = 0;
        // a group's views must fit above the tile bits of its keys (all-ones view: dead pairs)
        if (B.P.tbits > kTileBits) return fail(ctx, DGS_ERR_CAPACITY, "one view has 2^24 tiles or more");
        const int key_views = (int)std::min<int64_t>((1ll << (kTileBits - B.P.tbits)) - 1, V);
        const int cap_views = std::min(o.views_per_group > 0 ? o.views_per_group : V, std::max(key_views, 1));
        // automatic grouping of a large batch: two groups of about half the tile pairs each, so
        // that the second group's binning overlaps the first group's compositing
        int split_at = -1;
        if (o.views_per_group == 0 && V >= 2 && pair_at[V] >= kPipelinePairs) {
            split_at = 1;
            while (split_at < V - 1 && pair_at[split_at] < pair_at[V] / 2) ++split_at;
        }
        auto tile_end = [&](int v) { return v < V ? (int64_t)B.views[v].tile_base : B.tiles_total; };
        for (int v = 0; v < V; ++v) {
            if (pair_at[v + 1] - pair_at[v] > kMaxPairs)
                return fail(ctx, DGS_ERR_CAPACITY, "one view has more than 2^30 tile pairs");
            if (tile_end(v + 1) - tile_end(v) > kMaxGroupTiles)
                return fail(ctx, DGS_ERR_CAPACITY, "one view has 2^24 tiles or more");
            if (v > v0 && (pair_at[v + 1] - pair_at[v0] > kMaxPairs || tile_end(v + 1) - tile_end(v0) > kMaxGroupTiles ||
                           v - v0 >= cap_views || v == split_at)) {
                groups.push_back({v0, v});
                v0 = v;
            }
        }
        groups.push_back({v0, V});
    }
    uint64_t max_inst = 1, max_pairs = 1;
    int64_t max_tiles = 1;
    int max_bits = 0;
    for (auto& g : groups) {
        max_inst = std::max<uint64_t>(max_inst, inst_at[g.second] - inst_at[g.first]);
        max_pairs = std::max<uint64_t>(max_pairs, pair_at[g.second] - pair_at[g.first]);
        const int64_t t0 = B.views[g.first].tile_base;
        const int64_t t1 = g.second < V ? B.views[g.second].tile_base : B.tiles_total;
        max_tiles = std::max<int64_t>(max_tiles, t1 - t0);
        if (pair_at[g.second] - pair_at[g.first] > kMaxPairs)
            return fail(ctx, DGS_ERR_CAPACITY, "view group exceeds 2^30 tile pairs");
    }
    max_bits = B.P.tbits;                 // the tile sort radixes the tile-in-view bits only
    if (max_tiles > kMaxGroupTiles) return fail(ctx, DGS_ERR_CAPACITY, "more than 2^24 - 1 tiles in a view group");
    ctx->stats.n_groups = (int32_t)groups.size();
    ctx->stats.key_bits = max_bits;
    if (need) {   // a workspace query: the bytes of the lists, nothing allocated
        size_t bytes[ListBufs::kCount];
        list_bytes(max_inst, max_pairs, max_tiles, o.tile_w * o.tile_h, o.keep_lists != 0, bytes);
        size_t s = 0;
        for (size_t b : bytes) s += b;
        *need = s * (groups.size() > 1 ? 2 : 1);
        return DGS_OK;
    }
    if ((rc = ensure_lists(ctx, ctx->lists[0], max_inst, max_pairs, max_tiles))) return rc;
    if (groups.size() > 1 && (rc = ensure_lists(ctx, ctx->lists[1], max_inst, max_pairs, max_tiles))) return rc;
    B.groups = std::move(groups);
    B.inst_at = inst_at; B.pair_at = pair_at;
    return DGS_OK;
}

// The eager sequence's front half: staging, setup/count/scan and the readback.
int prepare(dgs_ctx* ctx, const dgs_node* nodes, int32_t n_nodes, const int32_t* env_node_ids, int32_t n_envs,
            int32_t max_nodes, const float* node_poses, const dgs_camera* cams, const int32_t* cams_per_env,
            int32_t max_cams, const float* out_rgb, const float* out_depth, const int64_t* view_pixel_offset,
            const dgs_node_grads* grads, cudaStream_t stream, Timer& tm, Batch& B) {
    int rc = stage(ctx, nodes, n_nodes, env_node_ids, n_envs, max_nodes, node_poses, cams, cams_per_env, max_cams,
                   out_rgb, out_depth, view_pixel_offset, grads, stream, tm, B);
    if (rc != DGS_OK || B.V == 0) return rc;
    Launch L{stream, &ctx->launches};
    launch_front(ctx, B, L, tm);
    return readback_groups(ctx, B, stream, tm);
}

// The depth-ordered tile lists of views [v0, v1): emission (K2), depth sort of the instances,
// pair offsets in depth order, pair emission, stable tile sort (K3) and tile ranges (K4).
//   n_inst   instances of the group (host count; the capacity when d_inst is set)
//   n_bound  bound on its pairs (host; the capacity the pair buffers hold)
//   d_inst   device count of instances (graph replay) or null
//   d_pairs  device word receiving the group's exact pair count (at most n_bound)
// Returns the tile-sorted instance numbers in *vals and, for groups of at most kOrderMaxTiles
// tiles, the tiles by descending list length in *tile_order (else null).  With want_ck and
// keep_lists, and room for them, *ck receives the checkpoints that the group's compositor is to
// write and the adjoint's (tile, segment) jobs (bounded by *n_jobs_bound); else ck->st is null.
void enqueue_lists(dgs_ctx* ctx, ListBufs& lb, const Batch& B, const Launch& L, Timer& tm, int v0, int v1, int n_tiles,
                   uint32_t inst_base, uint32_t n_inst, uint32_t n_bound, const uint32_t* d_inst, uint32_t* d_pairs,
                   const Params& P, const uint32_t** keys, const uint32_t** vals, const uint32_t** tile_order,
                   Checkpoints* ck, uint32_t* n_jobs_bound, bool want_ck = true) {
    const int K = B.K;
    auto u32 = [](DevBuf& b) { return static_cast<uint32_t*>(b.p); };
    Record* rec = static_cast<Record*>(lb.records.p);
    InstInfo* info = static_cast<InstInfo*>(lb.info.p);
    // the depth sort's view key: packed into the instance numbers where both fit in 32 bits
    ViewKey vk;
    vk.bits = bits_for((uint64_t)(v1 - v0));
    // (test_fault 4: the gathered form, as for groups whose numbers leave no room)
    if (vk.bits > 0 && bits_for((uint64_t)n_inst) + vk.bits <= 32 && ctx->opt.test_fault != 4)
        vk.vshift = 32 - vk.bits;
    vk.vig = vk.bits > 0 && !vk.vshift ? u32(lb.vig) : nullptr;
    vk.inst_off = B.d_inst_off;
    vk.view_tab = B.d_viewtab;
    vk.v0 = v0;
    vk.nv = v1 - v0;
    Params Pe = P;
    Pe.vshift = vk.vshift;
    tm.begin(DGS_K_EMIT);
    launch_emit(L, B.dtype_mask, B.d_nodes, B.n_nodes, B.d_views, B.d_vnodes, K, B.d_nv, B.d_nvoff, (int)B.chunk_total,
                Pe, v0, v1, B.batched, B.d_pmap + (size_t)v0 * (2 * K + 1), B.view_tab[v0 + 1] - B.view_tab[v0],
                B.d_counts, B.d_inst_off, inst_base, rec, info, u32(lb.dkey0), u32(lb.ival0), u32(lb.ntile),
                const_cast<uint32_t*>(vk.vig));
    tm.end();
    tm.begin(DGS_K_SORT);
    uint32_t *dk = nullptr, *order = nullptr;
    SortCtl ctl;
    if (ctx->opt.spin_limit_us > 0) ctl.spin_ns = (uint64_t)ctx->opt.spin_limit_us * 1000ull;
    SortCtl depth_ctl = ctl, tile_ctl = ctl;
    if (ctx->opt.test_fault == 1) depth_ctl.mute_part = 1;
    tile_ctl.runs = true;   // an instance's pairs are consecutive tiles of one view
    depth_ctl.runs = true;  // emission order (view by view, Z-ordered nodes) keeps the high depth digits in runs
    // instances by depth, then by view (most significant, through the values): each view's
    // instances in depth order, so that every instance's pairs come out view by view
    launch_sort(L, u32(lb.dkey0), u32(lb.ival0), u32(lb.dkey1), u32(lb.ival1), n_inst, kZBits, u32(lb.hist),
                u32(lb.status), u32(lb.counters), B.d_err, &dk, &order, d_inst, depth_ctl, &vk);
    launch_tile_scan(L, order, u32(lb.ntile), n_inst, d_inst, u32(lb.poff), u32(lb.tparts), n_bound, d_pairs, B.d_err);
    launch_pairs(L, B.d_views, K, order, u32(lb.poff), rec, info, n_inst, d_inst, P, u32(lb.tkeys0),
                 u32(lb.tvals0), n_bound);
    uint32_t *tk = nullptr, *tv = nullptr;
    // pairs by tile in view only: stability keeps them view by view within each tile index
    launch_sort(L, u32(lb.tkeys0), u32(lb.tvals0), u32(lb.tkeys1), u32(lb.tvals1), n_bound, P.tbits, u32(lb.hist),
                u32(lb.status), u32(lb.counters), B.d_err, &tk, &tv, d_pairs, tile_ctl);
    tm.end();
    tm.begin(DGS_K_RANGES);
    launch_ranges(L, tk, n_bound, static_cast<uint2*>(lb.ranges.p), n_tiles, d_pairs, B.d_views, v1 - v0, P);
    *tile_order = nullptr;
    if (n_tiles <= kOrderMaxTiles && lb.torder.bytes >= sizeof(uint32_t) * (size_t)n_tiles) {
        launch_tile_order(L, static_cast<uint2*>(lb.ranges.p), n_tiles, static_cast<uint32_t*>(lb.torder.p));
        *tile_order = static_cast<uint32_t*>(lb.torder.p);
    }
    *ck = Checkpoints{};
    *n_jobs_bound = 0;
    const size_t ck_need = ck_state_bytes(n_bound, n_tiles, P.tile_w * P.tile_h);
    if (want_ck && ctx->opt.keep_lists && ck_need && lb.ck_st.bytes >= ck_need) {
        ck->st = static_cast<CkState*>(lb.ck_st.p);
        ck->off = u32(lb.ck_off);
        ck->last = u32(lb.ck_last);
        ck->jobs = static_cast<uint2*>(lb.ck_jobs.p);
        ck->n_jobs = u32(lb.ck_njobs);
        *n_jobs_bound = (uint32_t)(n_tiles + ck_slots(n_bound));
        launch_segment_jobs(L, static_cast<uint2*>(lb.ranges.p), n_tiles, *ck);
    }
    tm.end();
    *keys = tk;
    *vals = tv;
}

// The lists of view group g (eager sequence, host-known sizes).
struct GroupLists {
    int v0 = 0, v1 = 0, n_tiles = 0;
    uint32_t n_bound = 0, n_inst = 0;
    const uint32_t* keys = nullptr;
    const uint32_t* vals = nullptr;
    const uint32_t* order = nullptr;      // tiles by descending list length, or null
    Checkpoints ck{};                     // compositor checkpoints (keep_lists), or ck.st null
    uint32_t n_jobs_bound = 0;            // bound on the adjoint's (tile, segment) jobs
    ListBufs* lb = nullptr;
    Params P{};
};

// dgs_options.keep_lists: what an eager render leaves for a backward of the same batch -- its
// staged batch (device tables and host copy), the per-view counts it read back, every view
// group's lists (records, identities, tile-sorted pairs, ranges; at most two groups, one per
// list workspace), and the signature of the call's host-visible arguments.
struct SavedForward {
    bool valid = false;
    std::vector<unsigned char> sig;
    Batch B;
    std::vector<uint64_t> inst_at, pair_at;
    std::vector<GroupLists> groups;
    dgs_stats stats{};
};

void invalidate_saved(dgs_ctx* ctx) {
    if (ctx->saved) ctx->saved->valid = false;
}

// Bytes of every host-visible argument the lists depend on: the node descriptors (pointers,
// sizes, types), the env -> node table, the node-pose pointer, the cameras, the per-env camera
// counts and the pixel offsets.
std::vector<unsigned char> call_signature(const dgs_node* nodes, int32_t n_nodes, const int32_t* env_node_ids,
                                          int32_t n_envs, int32_t max_nodes, const float* node_poses,
                                          const dgs_camera* cams, const int32_t* cams_per_env, int32_t max_cams,
                                          const int64_t* view_pixel_offset) {
    std::vector<unsigned char> sig;
    auto put = [&](const void* p, size_t n) {
        const unsigned char* c = static_cast<const unsigned char*>(p);
        if (c) sig.insert(sig.end(), c, c + n);
        else sig.insert(sig.end(), n, 0xFF);
    };
    const int32_t dims[4] = {n_nodes, n_envs, max_nodes, max_cams};
    put(dims, sizeof(dims));
    if (n_nodes < 0 || n_envs < 0 || max_nodes < 0 || max_cams < 0) return sig;
    put(nodes, sizeof(dgs_node) * (size_t)n_nodes);
    put(env_node_ids, sizeof(int32_t) * (size_t)n_envs * (size_t)max_nodes);
    put(&node_poses, sizeof(node_poses));
    put(cams, sizeof(dgs_camera) * (size_t)n_envs * (size_t)max_cams);
    put(cams_per_env, sizeof(int32_t) * (size_t)n_envs);
    int64_t V = 0;
    if (cams_per_env)
        for (int32_t e = 0; e < n_envs; ++e) V += std::min(std::max(cams_per_env[e], 0), max_cams);
    const unsigned char has = view_pixel_offset ? 1 : 0;
    put(&has, 1);
    if (view_pixel_offset) put(view_pixel_offset, sizeof(int64_t) * (size_t)V);
    return sig;
}

void build_group_lists(dgs_ctx* ctx, const Batch& B, int g, ListBufs& lb, cudaStream_t stream, Timer& tm,
                       GroupLists& G, bool for_forward = true) {
    Launch L{stream, &ctx->launches};
    const int V = B.V;
    const int v0 = B.groups[g].first, v1 = B.groups[g].second;
    G.v0 = v0; G.v1 = v1;
    G.n_bound = (uint32_t)(B.pair_at[v1] - B.pair_at[v0]);
    G.n_inst = (uint32_t)(B.inst_at[v1] - B.inst_at[v0]);
    const int32_t tile0 = B.views[v0].tile_base;
    G.n_tiles = (int)((v1 < V ? B.views[v1].tile_base : B.tiles_total) - tile0);
    G.P = B.P;
    G.P.tile0 = tile0;
    G.P.view0 = (uint32_t)v0;
    G.P.n_rec = G.n_inst;
    G.lb = &lb;
    enqueue_lists(ctx, lb, B, L, tm, v0, v1, G.n_tiles, (uint32_t)B.inst_at[v0], G.n_inst, G.n_bound, nullptr,
                  static_cast<uint32_t*>(ctx->totals.p) + g, G.P, &G.keys, &G.vals, &G.order, &G.ck,
                  &G.n_jobs_bound, for_forward);
    // test_fault 3 (debug builds): the compositors' bound on instance numbers is half the
    // records written, so the entries of the upper half fail the check while every access the
    // check lets through stays inside the records of the group
    if (ctx->opt.test_fault == 3) G.P.n_rec = G.n_inst / 2;
}

// dgs_options.check_binning: reads view group g's tile lists back and checks them on the host
// (Sec. III-A: every tile must receive, in depth order, the instances that reach it).  A
// violation synchronises the device and returns DGS_ERR_CUDA with a description.
int check_lists(dgs_ctx* ctx, const Batch& B, int g, const GroupLists& G, cudaStream_t s) {
    (void)B;
    uint32_t n = 0;
    DGS_CUDA(ctx, cudaMemcpyAsync(&n, static_cast<uint32_t*>(ctx->totals.p) + g, sizeof(uint32_t),
                                  cudaMemcpyDeviceToHost, s));
    DGS_CUDA(ctx, cudaStreamSynchronize(s));
    n = std::min(n, G.n_bound);
    std::vector<uint32_t> keys(n), vals(n);
    std::vector<uint2> ranges((size_t)std::max(G.n_tiles, 0));
    std::vector<Record> rec(G.n_inst);
    if (n) {
        DGS_CUDA(ctx, cudaMemcpy(keys.data(), G.keys, sizeof(uint32_t) * n, cudaMemcpyDeviceToHost));
        DGS_CUDA(ctx, cudaMemcpy(vals.data(), G.vals, sizeof(uint32_t) * n, cudaMemcpyDeviceToHost));
    }
    if (!ranges.empty())
        DGS_CUDA(ctx, cudaMemcpy(ranges.data(), G.lb->ranges.p, sizeof(uint2) * ranges.size(), cudaMemcpyDeviceToHost));
    if (!rec.empty())
        DGS_CUDA(ctx, cudaMemcpy(rec.data(), G.lb->records.p, sizeof(Record) * rec.size(), cudaMemcpyDeviceToHost));
    if (ctx->opt.test_fault == 2 && g == 0)
        for (uint32_t i = 0; i + 1 < n; ++i)
            if ((keys[i] & kTileMask) != (keys[i + 1] & kTileMask)) {
                std::swap(keys[i], keys[i + 1]);
                std::swap(vals[i], vals[i + 1]);
                break;
            }
    const uint32_t n_sub = (uint32_t)(ctx->opt.tile_w * ctx->opt.tile_h / 32);
    std::string why;
    auto bad = [&](const std::string& what, uint64_t i) {
        why = "binning invariant violated in view group " + std::to_string(g) + ": " + what + " at pair " +
              std::to_string(i);
        return false;
    };
    // a key names (view in the group, tile in that view): sorted by tile in view, then view
    const int tb = G.P.tbits, nv = G.v1 - G.v0;
    const int64_t tile0 = B.views[G.v0].tile_base;
    const uint32_t tmask = (1u << tb) - 1u;
    auto group_tile = [&](uint32_t key) -> int64_t {   // tile in the group, -1 if none
        const uint32_t f = key & kTileMask, vg = f >> tb, ti = f & tmask;
        if (vg >= (uint32_t)nv) return -1;
        const ViewDesc& vd = B.views[G.v0 + vg];
        if (ti >= (uint32_t)(vd.tiles_x * vd.tiles_y)) return -1;
        return vd.tile_base - tile0 + ti;
    };
    auto order_key = [&](uint32_t key) { return ((uint64_t)(key & tmask) << 32) | ((key & kTileMask) >> tb); };
    auto check = [&]() {
        uint64_t covered = 0;
        for (uint32_t i = 0; i < n; ++i) {
            const uint32_t m = keys[i] >> kTileBits;
            if (group_tile(keys[i]) < 0) return bad("tile beyond the group", i);
            if (i && order_key(keys[i]) < order_key(keys[i - 1])) return bad("tiles not in order", i);
            // an empty mask is valid: the ellipse meets the tile's rectangle of pixel centres only
            // between two rows or columns of them, so no warp stages the pair
            if (m >= (1u << n_sub)) return bad("sub-tile mask", i);
            if (vals[i] >= G.n_inst) return bad("instance beyond the group", i);
        }
        for (int t = 0; t < G.n_tiles; ++t) {
            const uint2 r = ranges[t];
            if (r.x == r.y) continue;
            if (r.x > r.y || r.y > n) return bad("range of tile " + std::to_string(t), r.x);
            if ((r.x > 0 && group_tile(keys[r.x - 1]) == t) || (r.y < n && group_tile(keys[r.y]) == t))
                return bad("range of tile " + std::to_string(t) + " not maximal", r.x);
            for (uint32_t i = r.x; i < r.y; ++i) {
                if (group_tile(keys[i]) != t) return bad("range of tile " + std::to_string(t), i);
                if (i > r.x) {
                    const float z0 = rec[vals[i - 1]].r0.w, z1 = rec[vals[i]].r0.w;
                    if (z1 < z0 || (z1 == z0 && vals[i] <= vals[i - 1])) return bad("depth order in a tile", i);
                }
            }
            covered += r.y - r.x;
        }
        if (covered != n) return bad("ranges cover " + std::to_string(covered) + " of the pairs", n);
        return true;
    };
    if (check()) return DGS_OK;
    cudaDeviceSynchronize();
    return fail(ctx, DGS_ERR_CUDA, why);
}

// Final synchronisation, device error word and kernel times.
int finish(dgs_ctx* ctx, const Batch& B, cudaStream_t stream) {
    uint32_t* h_err = reinterpret_cast<uint32_t*>(static_cast<char*>(ctx->h_read) + sizeof(uint64_t) * 2 * (B.V + 1));
    uint32_t* h_tot = reinterpret_cast<uint32_t*>(static_cast<char*>(ctx->h_read) + sizeof(uint64_t) * 2 * (B.V + 1) + 64);
    const size_t ng = B.groups.size();
    DGS_CUDA(ctx, cudaGetLastError());
    DGS_CUDA(ctx, cudaMemcpyAsync(h_err, B.d_err, sizeof(uint32_t), cudaMemcpyDeviceToHost, stream));
    if (ng) DGS_CUDA(ctx, cudaMemcpyAsync(h_tot, ctx->totals.p, sizeof(uint32_t) * ng, cudaMemcpyDeviceToHost, stream));
    DGS_CUDA(ctx, cudaStreamSynchronize(stream));
    const uint32_t errw = *h_err;
    int64_t pairs = 0;
    for (size_t g = 0; g < ng; ++g) pairs += h_tot[g];
    ctx->stats.n_pairs = pairs;
    if (ctx->opt.profile) {
        for (const TimedRange& r : ctx->ranges_timed) {
            float ms = 0.f;
            if (cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) ctx->ktimes[r.cls] += ms;
        }
    }
    if (errw & kErrBounds) return bounds_failure(ctx, B.d_err);
    if (errw & kErrTimeout) return fail(ctx, DGS_ERR_TIMEOUT, "a bounded device wait timed out (sort look-back)");
    if (errw & kErrMismatch) return fail(ctx, DGS_ERR_CUDA, "internal: count and emit passes disagree");
    if (errw & kErrCapacity) return fail(ctx, DGS_ERR_CUDA, "internal: tile pairs beyond their bound");
    if (errw & kErrPose) return fail(ctx, DGS_ERR_INVALID_ARG, "a node pose is not finite or not rigid");
    return DGS_OK;
}

// ------------------------------------------------------------------ eager sequence
// Setup/count/scan, the readback, then per view group emit/sort/ranges/composite, and the
// final synchronisation.  B must have been staged.
int run_eager(dgs_ctx* ctx, Batch& B, float* out_rgb, float* out_depth, float* out_alpha, cudaStream_t stream,
              Timer& tm, std::vector<GroupLists>* keep = nullptr) {
    Launch L{stream, &ctx->launches};
    launch_front(ctx, B, L, tm);
    int rc = readback_groups(ctx, B, stream, tm);
    if (rc != DGS_OK) return rc;
    unsigned long long* work = nullptr;
    if (ctx->opt.profile >= 2) {
        work = reinterpret_cast<unsigned long long*>(static_cast<char*>(ctx->errword.p) + 32);
        DGS_CUDA(ctx, cudaMemsetAsync(work, 0, 24, stream));
    }
    // view groups alternate between the caller's stream and a second one, each with its own
    // list workspace, so one group's binning overlaps the previous group's compositing
    const int ng = (int)B.groups.size();
    cudaStream_t streams[2] = {stream, stream};
    if (ng > 1) {
        if (!ctx->aux_stream) DGS_CUDA(ctx, cudaStreamCreateWithFlags(&ctx->aux_stream, cudaStreamNonBlocking));
        streams[1] = ctx->aux_stream;
        cudaEvent_t front = take_event(ctx);
        DGS_CUDA(ctx, cudaEventRecord(front, stream));
        DGS_CUDA(ctx, cudaStreamWaitEvent(streams[1], front, 0));
    }
    Timer tms[2] = {tm, Timer{ctx, streams[1], tm.on}};
    for (int g = 0; g < ng; ++g) {
        const int b = g & 1;
        GroupLists G;
        build_group_lists(ctx, B, g, ctx->lists[b], streams[b], tms[b], G);
        if (ctx->opt.check_binning && (rc = check_lists(ctx, B, g, G, streams[b]))) return rc;
        Launch Lg{streams[b], &ctx->launches};
        tms[b].begin(DGS_K_COMPOSITE);
        launch_composite(Lg, B.d_views, G.v0, G.v1 - G.v0, G.n_tiles, static_cast<uint2*>(G.lb->ranges.p), G.keys, G.vals,
                         static_cast<Record*>(G.lb->records.p), G.P, out_rgb, out_depth, out_alpha, work, G.order,
                         G.ck);
        tms[b].end();
        DGS_CUDA(ctx, cudaGetLastError());
        if (keep) keep->push_back(G);
    }
    if (ng > 1) {
        cudaEvent_t join = take_event(ctx);
        DGS_CUDA(ctx, cudaEventRecord(join, streams[1]));
        DGS_CUDA(ctx, cudaStreamWaitEvent(stream, join, 0));
    }
    rc = finish(ctx, B, stream);
    if (rc == DGS_OK && work) {
        unsigned long long h[3] = {0, 0, 0};
        DGS_CUDA(ctx, cudaMemcpy(h, work, sizeof(h), cudaMemcpyDeviceToHost));
        ctx->stats.px_evaluated = (int64_t)h[0];
        ctx->stats.px_reached = (int64_t)h[1];
        ctx->stats.px_composited = (int64_t)h[2];
    }
    return rc;
}

// ------------------------------------------------------------------ graph replay
// The captured sequence runs one or two view groups; group g covers views [v0, v1) whose
// count-table entries are [t0, t1).
struct GraphGroups {
    int64_t t0[2], t1[2];
    uint64_t cap_inst[2], cap_pairs[2];
    const ulonglong2* scan_total;         // 64-bit totals of the count scan (null: no entries)
    int32_t ng;
};

// gsizes layout (u32 words): group g at [8g]: [8g] live instances, [8g+1] live pair bound,
// [8g+3] exact pairs (written by the tile-count scan), [8g+4] the group's first record; [2]
// the overflow flag of the whole replay; u64 at word 16: the instance and pair-bound totals of
// each group (valid even on overflow).
__global__ void k_graph_sizes(const uint32_t* __restrict__ inst_off, const uint64_t* __restrict__ pair_off,
                              GraphGroups G, uint32_t* sizes, uint32_t* err) {
    uint64_t ni[2] = {0, 0}, np[2] = {0, 0};
    // the 32-bit instance offsets wrap at 2^32: the scan's 64-bit total decides first
    bool over = G.scan_total && G.scan_total->x >= (1ull << 32);
    for (int g = 0; g < G.ng; ++g) {
        ni[g] = (uint64_t)inst_off[G.t1[g]] - inst_off[G.t0[g]];
        np[g] = pair_off[G.t1[g]] - pair_off[G.t0[g]];
        over |= ni[g] > G.cap_inst[g] || np[g] > G.cap_pairs[g];
    }
    uint64_t* raw = reinterpret_cast<uint64_t*>(sizes + 16);
    for (int g = 0; g < 2; ++g) {
        uint32_t* s = sizes + 8 * g;
        s[0] = over ? 0u : (uint32_t)ni[g];
        s[1] = over ? 0u : (uint32_t)np[g];
        s[3] = 0u;
        s[4] = g < G.ng ? inst_off[G.t0[g]] : 0u;
        raw[2 * g] = ni[g];
        raw[2 * g + 1] = np[g];
    }
    sizes[2] = over ? 1u : 0u;
    if (over) atomicOr(err, kErrCapacity);
}

GraphKey make_key(const dgs_ctx* ctx, const Batch& B, const float* rgb, const float* depth, const float* alpha) {
    GraphKey k;
    std::memset(&k, 0, sizeof(k));
    k.V = B.V; k.K = B.K; k.n_nodes = B.n_nodes; k.dtype_mask = B.dtype_mask; k.chunk_total = B.chunk_total;
    k.T = B.T; k.tiles_total = B.tiles_total; k.n_nv = B.n_nv; k.upload_bytes = (int64_t)B.upload_bytes;
    k.meta_bytes = (int64_t)B.meta_bytes;
    k.poses = B.node_poses; k.rgb = rgb; k.depth = depth; k.alpha = alpha;
    k.gen = ctx->gen;
    k.tile_w = ctx->opt.tile_w; k.tile_h = ctx->opt.tile_h; k.exact_tile_test = ctx->opt.exact_tile_test;
    k.ng = ctx->gng; k.split = ctx->gsplit;
    k.overlay = ctx->overlay;
    k.aug_on = !ctx->aug.empty(); k.ov_n = ctx->ov_n; k.ov_w = ctx->ov_w; k.ov_h = ctx->ov_h;
    return k;
}

bool same_key(const GraphKey& a, const GraphKey& b) { return std::memcmp(&a, &b, sizeof(a)) == 0; }

void drop_graph(dgs_ctx* ctx) {
    if (ctx->gexec) cudaGraphExecDestroy(ctx->gexec);
    ctx->gexec = nullptr;
}

// The whole render as one sequence sized for the context's capacities; every kernel after the
// scan reads the live counts on the device, so nothing is read back between count and
// composite.  With two view groups the second runs on a forked stream (its binning overlaps
// the first group's compositing) and joins before the end.  On overflow the size check raises
// kErrCapacity and the later kernels do no work.
int enqueue_graph_body(dgs_ctx* ctx, const Batch& B, const Launch& L, float* out_rgb, float* out_depth,
                       float* out_alpha) {
    Timer off{ctx, L.stream, false};
    launch_front(ctx, B, L, off);
    uint32_t* sizes = static_cast<uint32_t*>(ctx->gsizes.p);
    const int ng = ctx->gng;
    const int vb[3] = {0, ng == 2 ? ctx->gsplit : B.V, B.V};
    GraphGroups G{};
    G.ng = ng;
    G.scan_total = B.n_parts > 0 ? static_cast<ulonglong2*>(ctx->parts.p) + B.n_parts : nullptr;
    for (int g = 0; g < ng; ++g) {
        G.t0[g] = B.view_tab[vb[g]];
        G.t1[g] = B.view_tab[vb[g + 1]];
        G.cap_inst[g] = ctx->cap_inst[g];
        G.cap_pairs[g] = ctx->cap_pairs[g];
    }
    k_graph_sizes<<<1, 1, 0, L.stream>>>(B.d_inst_off, B.d_pair_off, G, sizes, B.d_err);
    ++*L.launches;
    cudaStream_t st[2] = {L.stream, ctx->cap_stream2};
    if (ng == 2) {
        cudaEvent_t fork = take_event(ctx);
        DGS_CUDA(ctx, cudaEventRecord(fork, L.stream));
        DGS_CUDA(ctx, cudaStreamWaitEvent(st[1], fork, 0));
    }
    for (int g = 0; g < ng; ++g) {
        const int v0 = vb[g], v1 = vb[g + 1];
        const int32_t tile0 = B.views[v0].tile_base;
        const int n_tiles = (int)((v1 < B.V ? B.views[v1].tile_base : B.tiles_total) - tile0);
        Launch Lg{st[g], L.launches};
        Timer tg{ctx, st[g], false};
        Params P = B.P;
        P.tile0 = tile0;
        P.gate = sizes + 2;
        P.inst_base_dev = sizes + 8 * g + 4;
        P.n_rec = (uint32_t)ctx->cap_inst[g];
        P.view0 = (uint32_t)v0;
        ListBufs& lb = ctx->lists[g];
        const uint32_t *keys = nullptr, *vals = nullptr, *order = nullptr;
        Checkpoints ck{};
        uint32_t n_jobs_bound = 0;
        enqueue_lists(ctx, lb, B, Lg, tg, v0, v1, n_tiles, 0u, (uint32_t)ctx->cap_inst[g],
                      (uint32_t)ctx->cap_pairs[g], sizes + 8 * g, sizes + 8 * g + 3, P, &keys, &vals, &order, &ck,
                      &n_jobs_bound);
        launch_composite(Lg, B.d_views, v0, v1 - v0, n_tiles, static_cast<uint2*>(lb.ranges.p), keys, vals,
                         static_cast<Record*>(lb.records.p), P, out_rgb, out_depth, out_alpha, nullptr, order, ck);
        ctx->gv0[g] = v0; ctx->gv1[g] = v1; ctx->gtiles[g] = n_tiles;
        ctx->gkeys[g] = keys; ctx->gvals[g] = vals; ctx->gorder[g] = order; ctx->gP[g] = P;
        ctx->gck[g] = ck; ctx->gjobs[g] = n_jobs_bound;
    }
    if (ng == 2) {
        cudaEvent_t join = take_event(ctx);
        DGS_CUDA(ctx, cudaEventRecord(join, st[1]));
        DGS_CUDA(ctx, cudaStreamWaitEvent(L.stream, join, 0));
    }
    return DGS_OK;
}

// Captures the sequence with the view groups of the eager render just done (B: one or two
// groups) and capacities of 1.25x its per-group instance and pair-bound totals.  Returns
// DGS_OK without a graph when the batch needs more than two groups or a group more than 2^31
// tiles.
int capture_graph(dgs_ctx* ctx, const Batch& B, float* out_rgb, float* out_depth, float* out_alpha) {
    drop_graph(ctx);
    const int ng = (int)B.groups.size();
    if (ng < 1 || ng > 2) return DGS_OK;
    const int split = ng == 2 ? B.groups[0].second : B.V;
    const bool same_split = ng == ctx->gng && split == ctx->gsplit;
    ctx->gng = ng;
    ctx->gsplit = split;
    int rc;
    int bits = 0;
    for (int g = 0; g < ng; ++g) {
        const int v0 = B.groups[g].first, v1 = B.groups[g].second;
        const uint64_t need_inst = B.inst_at[v1] - B.inst_at[v0], need_pairs = B.pair_at[v1] - B.pair_at[v0];
        const int64_t n_tiles = (v1 < B.V ? B.views[v1].tile_base : B.tiles_total) - B.views[v0].tile_base;
        bits = B.P.tbits;
        if (need_pairs > kMaxPairs || n_tiles > kMaxGroupTiles || need_inst >= (1ull << 31)) return DGS_OK;
        const uint64_t ci = need_inst + need_inst / 4 + 1024;
        const uint64_t cp = std::min<uint64_t>(kMaxPairs, need_pairs + need_pairs / 4 + 4096);
        ctx->cap_inst[g] = same_split ? std::max(ctx->cap_inst[g], ci) : ci;
        ctx->cap_pairs[g] = same_split ? std::max(ctx->cap_pairs[g], cp) : cp;
        if ((rc = ensure_lists(ctx, ctx->lists[g], ctx->cap_inst[g], ctx->cap_pairs[g], n_tiles))) return rc;
    }
    ctx->gbits = bits;
    if ((rc = ensure(ctx, ctx->gsizes, 128))) return rc;
    if (!ctx->h_graph) DGS_CUDA(ctx, cudaHostAlloc(&ctx->h_graph, 128, cudaHostAllocDefault));
    if (!ctx->cap_stream) DGS_CUDA(ctx, cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking));
    if (!ctx->cap_stream2) DGS_CUDA(ctx, cudaStreamCreateWithFlags(&ctx->cap_stream2, cudaStreamNonBlocking));
    sort_prepare();
    int64_t n_launch = 0;
    Launch L{ctx->cap_stream, &n_launch};
    DGS_CUDA(ctx, cudaStreamBeginCapture(ctx->cap_stream, cudaStreamCaptureModeThreadLocal));
    const int rb = enqueue_graph_body(ctx, B, L, out_rgb, out_depth, out_alpha);
    cudaGraph_t g = nullptr;
    const cudaError_t e = cudaStreamEndCapture(ctx->cap_stream, &g);
    if (rb != DGS_OK || e != cudaSuccess || !g) {
        cudaGetLastError();
        if (g) cudaGraphDestroy(g);
        if (rb != DGS_OK) return rb;
        return cuda_fail(ctx, e != cudaSuccess ? e : cudaErrorUnknown, "stream capture of the render sequence");
    }
    const cudaError_t ei = cudaGraphInstantiate(&ctx->gexec, g, 0);
    cudaGraphDestroy(g);
    if (ei != cudaSuccess) {
        ctx->gexec = nullptr;
        cudaGetLastError();
        return cuda_fail(ctx, ei, "cudaGraphInstantiate");
    }
    ctx->gkey = make_key(ctx, B, out_rgb, out_depth, out_alpha);
    ctx->glaunches = n_launch;
    ++ctx->captures;
    return DGS_OK;
}

// DGS_MODE_GRAPH: replay the captured sequence when the staged batch has the captured
// structure; otherwise (or after an overflow) render eagerly and capture for the next call.
int render_graph(dgs_ctx* ctx, Batch& B, float* out_rgb, float* out_depth, float* out_alpha, cudaStream_t stream,
                 Timer& tm, std::vector<GroupLists>* keep = nullptr) {
    int rc;
    if (ctx->gexec && same_key(make_key(ctx, B, out_rgb, out_depth, out_alpha), ctx->gkey)) {
        cudaEvent_t a = nullptr;
        if (ctx->opt.profile) {
            a = take_event(ctx);
            cudaEventRecord(a, stream);
        }
        DGS_CUDA(ctx, cudaGraphLaunch(ctx->gexec, stream));
        if (ctx->opt.profile) {
            cudaEvent_t b = take_event(ctx);
            cudaEventRecord(b, stream);
            ctx->ranges_timed.push_back({DGS_K_GRAPH, a, b});
        }
        ctx->launches = ctx->glaunches;
        char* hg = static_cast<char*>(ctx->h_graph);
        DGS_CUDA(ctx, cudaMemcpyAsync(hg, ctx->gsizes.p, 96, cudaMemcpyDeviceToHost, stream));
        DGS_CUDA(ctx, cudaMemcpyAsync(hg + 96, B.d_err, sizeof(uint32_t), cudaMemcpyDeviceToHost, stream));
        DGS_CUDA(ctx, cudaStreamSynchronize(stream));
        uint32_t errw, sizes[16];
        uint64_t raw[4];
        std::memcpy(sizes, hg, 64);
        std::memcpy(raw, hg + 64, 32);
        std::memcpy(&errw, hg + 96, 4);
        if (ctx->opt.profile)
            for (const TimedRange& r : ctx->ranges_timed) {
                float ms = 0.f;
                if (cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) ctx->ktimes[r.cls] += ms;
            }
        ctx->stats.n_visible = (int64_t)(raw[0] + raw[2]);
        ctx->stats.n_pairs = (int64_t)sizes[3] + (ctx->gng == 2 ? (int64_t)sizes[11] : 0);
        ctx->stats.n_groups = ctx->gng;
        ctx->stats.key_bits = ctx->gbits;
        if (errw & kErrPose) return fail(ctx, DGS_ERR_INVALID_ARG, "a node pose is not finite or not rigid");
        if (errw & kErrBounds) return bounds_failure(ctx, B.d_err);
        if (errw & kErrTimeout) return fail(ctx, DGS_ERR_TIMEOUT, "a bounded device wait timed out (sort look-back)");
        if (errw & kErrMismatch) return fail(ctx, DGS_ERR_CUDA, "internal: count and emit passes disagree");
        if (!(errw & kErrCapacity) || !sizes[2]) {
            if (errw & kErrCapacity) return fail(ctx, DGS_ERR_CUDA, "internal: tile pairs beyond their bound");
            ctx->stats.path = DGS_PATH_GRAPH;
            ctx->stats.graph_captures = ctx->captures;
            for (int g = 0; keep && g < ctx->gng; ++g) {
                GroupLists G;
                G.v0 = ctx->gv0[g]; G.v1 = ctx->gv1[g]; G.n_tiles = ctx->gtiles[g];
                G.n_bound = (uint32_t)ctx->cap_pairs[g];
                G.n_inst = (uint32_t)raw[2 * g];      // the replay's live count (at most the capacity)
                G.keys = ctx->gkeys[g]; G.vals = ctx->gvals[g]; G.order = ctx->gorder[g];
                G.ck = ctx->gck[g]; G.n_jobs_bound = ctx->gjobs[g];
                G.lb = &ctx->lists[g];
                G.P = ctx->gP[g];
                keep->push_back(G);
            }
            return DGS_OK;
        }
        // the replay's outputs are invalid: render again eagerly (the staged tables are still
        // in place) and capture with capacities sized for these totals
        ctx->ranges_timed.clear();
        ctx->launches = 0;
        if ((rc = run_eager(ctx, B, out_rgb, out_depth, out_alpha, stream, tm))) return rc;
        if ((rc = capture_graph(ctx, B, out_rgb, out_depth, out_alpha))) return rc;
        ctx->stats.path = DGS_PATH_REGROWN;
        return DGS_OK;
    }
    if ((rc = run_eager(ctx, B, out_rgb, out_depth, out_alpha, stream, tm))) return rc;
    if ((rc = capture_graph(ctx, B, out_rgb, out_depth, out_alpha))) return rc;
    ctx->stats.path = ctx->gexec ? DGS_PATH_CAPTURED : DGS_PATH_EAGER;
    return DGS_OK;
}

void begin_call(dgs_ctx* ctx) {
    ctx->err.clear();
    ctx->launches = 0;
    ctx->ranges_timed.clear();
    ctx->next_event = 0;
    for (float& t : ctx->ktimes) t = 0.f;
}

}  // namespace

extern "C" {

void dgs_default_options(dgs_options* o) {
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->mode = DGS_MODE_BATCHED;
    o->tile_w = 16;
    o->tile_h = 16;
    o->exact_tile_test = 1;
    o->z_near = 0.01f;
    o->lowpass = 0.3f;
    o->alpha_min = 1.0f / 255.0f;
    o->alpha_max = 0.99f;
    o->t_min = 1e-4f;
    o->q_max = 9.0f;
    o->guard = 1.3f;
    o->profile = 0;
    o->views_per_group = 0;
}

int dgs_context_create(dgs_ctx** out, const dgs_options* opt) {
    if (!out) return DGS_ERR_INVALID_ARG;
    *out = nullptr;
    dgs_options o;
    if (opt) o = *opt; else dgs_default_options(&o);
    std::string why;
    if (!check_options(&o, why)) return DGS_ERR_INVALID_ARG;
    dgs_ctx* ctx = new dgs_ctx();
    ctx->opt = o;
    cudaGetDevice(&ctx->device);
    *out = ctx;
    return DGS_OK;
}

int dgs_set_options(dgs_ctx* ctx, const dgs_options* opt) {
    if (!ctx || !opt) return DGS_ERR_INVALID_ARG;
    std::string why;
    if (!check_options(opt, why)) return fail(ctx, DGS_ERR_INVALID_ARG, "options: " + why);
    ctx->opt = *opt;
    drop_graph(ctx);      // captured kernels carry the old options
    invalidate_saved(ctx);
    return DGS_OK;
}

int dgs_context_destroy(dgs_ctx* ctx) {
    if (!ctx) return DGS_OK;
    cudaDeviceSynchronize();
    DevBuf* bufs[] = {&ctx->meta, &ctx->counts, &ctx->inst_off, &ctx->pair_off, &ctx->parts, &ctx->errword,
                      &ctx->readback, &ctx->inst_grad, &ctx->gsizes, &ctx->totals};
    for (DevBuf* b : bufs) free_buf(*b);
    for (ListBufs& lb : ctx->lists)
        for (DevBuf* b : lb.all) free_buf(*b);
    if (ctx->aux_stream) cudaStreamDestroy(ctx->aux_stream);
    drop_graph(ctx);
    if (ctx->cap_stream) cudaStreamDestroy(ctx->cap_stream);
    if (ctx->cap_stream2) cudaStreamDestroy(ctx->cap_stream2);
    if (ctx->h_graph) cudaFreeHost(ctx->h_graph);
    if (ctx->h_meta) cudaFreeHost(ctx->h_meta);
    if (ctx->h_read) cudaFreeHost(ctx->h_read);
    free_buf(ctx->aug_dev);
    free_buf(ctx->tsdf_meta);
    free_buf(ctx->tsdf_depth);
    if (ctx->h_tsdf) cudaFreeHost(ctx->h_tsdf);
    if (ctx->tsdf_copied) cudaEventDestroy(ctx->tsdf_copied);
    for (DevBuf* b : {&ctx->lid_rec, &ctx->lid_box, &ctx->lid_tab, &ctx->lid_meta, &ctx->lid_slots}) free_buf(*b);
    if (ctx->h_lid) cudaFreeHost(ctx->h_lid);
    if (ctx->h_aug) cudaFreeHost(ctx->h_aug);
    if (ctx->aug_copied) cudaEventDestroy(ctx->aug_copied);
    for (cudaEvent_t e : ctx->events) cudaEventDestroy(e);
    delete ctx;
    return DGS_OK;
}

const char* dgs_last_error(const dgs_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

int dgs_workspace_query(const dgs_ctx* ctx, size_t* bytes) {
    if (!ctx || !bytes) return DGS_ERR_INVALID_ARG;
    const DevBuf* bufs[] = {&ctx->meta, &ctx->counts, &ctx->inst_off, &ctx->pair_off, &ctx->parts, &ctx->errword,
                            &ctx->readback, &ctx->inst_grad, &ctx->gsizes, &ctx->totals, &ctx->aug_dev,
                            &ctx->lid_rec, &ctx->lid_box, &ctx->lid_tab, &ctx->lid_meta, &ctx->lid_slots,
                            &ctx->tsdf_meta, &ctx->tsdf_depth};
    size_t s = 0;
    for (const DevBuf* b : bufs) s += b->bytes;
    for (const ListBufs& lb : ctx->lists)
        for (const DevBuf* b : lb.all) s += b->bytes;
    *bytes = s;
    return DGS_OK;
}

int dgs_workspace_query_batch(dgs_ctx* ctx, const dgs_node* nodes, int32_t n_nodes, const int32_t* env_node_ids,
                              int32_t n_envs, int32_t max_nodes, const float* node_poses, const dgs_camera* cams,
                              const int32_t* cams_per_env, int32_t max_cams, const int64_t* view_pixel_offset,
                              size_t* bytes, void* stream_) {
    if (!ctx) return DGS_ERR_INVALID_ARG;
    begin_call(ctx);
    if (!bytes) return fail(ctx, DGS_ERR_INVALID_ARG, "bytes is required");
    *bytes = 0;
    cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_);
    Timer tm{ctx, stream, false};
    Batch B;
    int rc = stage(ctx, nodes, n_nodes, env_node_ids, n_envs, max_nodes, node_poses, cams, cams_per_env, max_cams,
                   nullptr, nullptr, view_pixel_offset, nullptr, stream, tm, B, false);
    if (rc != DGS_OK || B.V == 0) return rc;
    Launch L{stream, &ctx->launches};
    launch_front(ctx, B, L, tm);
    size_t lists = 0;
    if ((rc = readback_groups(ctx, B, stream, tm, &lists))) return rc;
    *bytes = B.front_bytes + lists;
    return DGS_OK;
}

int dgs_last_stats(const dgs_ctx* ctx, dgs_stats* out) {
    if (!ctx || !out) return DGS_ERR_INVALID_ARG;
    *out = ctx->stats;
    return DGS_OK;
}

int dgs_kernel_times(const dgs_ctx* ctx, float* ms) {
    if (!ctx || !ms) return DGS_ERR_INVALID_ARG;
    for (int i = 0; i < DGS_K_COUNT_CLASSES; ++i) ms[i] = ctx->ktimes[i];
    return DGS_OK;
}

int64_t dgs_last_launches(const dgs_ctx* ctx) { return ctx ? ctx->launches : -1; }

int32_t dgs_build_flags(void) { return kDebugChecks ? DGS_BUILD_DEBUG : 0; }


int dgs_render(dgs_ctx* ctx, const dgs_node* nodes, int32_t n_nodes, const int32_t* env_node_ids, int32_t n_envs,
               int32_t max_nodes, const float* node_poses, const dgs_camera* cams, const int32_t* cams_per_env,
               int32_t max_cams, float* out_rgb, float* out_depth, float* out_alpha,
               const int64_t* view_pixel_offset, void* stream_) {
    if (!ctx) return DGS_ERR_INVALID_ARG;
    begin_call(ctx);
    cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_);
    Timer tm{ctx, stream, ctx->opt.profile != 0};
    Batch B;
    int rc = stage(ctx, nodes, n_nodes, env_node_ids, n_envs, max_nodes, node_poses, cams, cams_per_env, max_cams,
                   out_rgb, out_depth, view_pixel_offset, nullptr, stream, tm, B);
    if (rc != DGS_OK || B.V == 0) return rc;
    // keep_lists: the lists of at most two view groups (one per list workspace) stay in place;
    // an eager render keeps them, and so does a graph replay (not the call that captures)
    std::vector<GroupLists> groups;
    std::vector<GroupLists>* keep = ctx->opt.keep_lists ? &groups : nullptr;
    if (ctx->opt.mode == DGS_MODE_GRAPH && B.T > 0)
        rc = render_graph(ctx, B, out_rgb, out_depth, out_alpha, stream, tm, keep);
    else
        rc = run_eager(ctx, B, out_rgb, out_depth, out_alpha, stream, tm, keep);
    if (rc == DGS_OK && keep && !groups.empty() && groups.size() <= 2) {
        if (!ctx->saved) ctx->saved.reset(new SavedForward);
        SavedForward& S = *ctx->saved;
        S.sig = call_signature(nodes, n_nodes, env_node_ids, n_envs, max_nodes, node_poses, cams, cams_per_env,
                               max_cams, view_pixel_offset);
        S.B = B;
        S.inst_at.clear();
        S.pair_at.clear();
        if (B.inst_at) {
            S.inst_at.assign(B.inst_at, B.inst_at + B.V + 1);
            S.pair_at.assign(B.pair_at, B.pair_at + B.V + 1);
        }
        S.B.inst_at = B.inst_at ? S.inst_at.data() : nullptr;
        S.B.pair_at = B.pair_at ? S.pair_at.data() : nullptr;
        S.groups = std::move(groups);
        S.stats = ctx->stats;
        S.valid = true;
    }
    ctx->stats.graph_captures = ctx->captures;
    return rc;
}

int dgs_autotune(dgs_ctx* ctx, const dgs_node* nodes, int32_t n_nodes, const int32_t* env_node_ids, int32_t n_envs,
                 int32_t max_nodes, const float* node_poses, const dgs_camera* cams, const int32_t* cams_per_env,
                 int32_t max_cams, float* out_rgb, float* out_depth, float* out_alpha,
                 const int64_t* view_pixel_offset, const int32_t* candidates, int32_t n_candidates, int32_t reps,
                 dgs_tune_result* out, void* stream_) {
    if (!ctx) return DGS_ERR_INVALID_ARG;
    static const int32_t kDefault[5][2] = {{16, 16}, {32, 8}, {8, 32}, {16, 8}, {8, 8}};
    const int32_t* cand = candidates ? candidates : &kDefault[0][0];
    const int nc = candidates ? n_candidates : 5;
    if (!out) return fail(ctx, DGS_ERR_INVALID_ARG, "out is required");
    if (nc < 1 || nc > DGS_TUNE_MAX) return fail(ctx, DGS_ERR_INVALID_ARG, "n_candidates must be 1..16");
    if (reps < 1 || reps > 1000) return fail(ctx, DGS_ERR_INVALID_ARG, "reps must be 1..1000");
    for (int i = 0; i < nc; ++i) {
        dgs_options o = ctx->opt;
        o.tile_w = cand[2 * i];
        o.tile_h = cand[2 * i + 1];
        std::string why;
        if (!check_options(&o, why)) return fail(ctx, DGS_ERR_INVALID_ARG, "candidate " + std::to_string(i) + ": " + why);
    }
    cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_);
    const dgs_options saved = ctx->opt;
    cudaEvent_t a = nullptr, b = nullptr;
    DGS_CUDA(ctx, cudaEventCreate(&a));
    if (cudaEventCreate(&b) != cudaSuccess) {
        cudaEventDestroy(a);
        return fail(ctx, DGS_ERR_CUDA, "cudaEventCreate");
    }
    std::memset(out, 0, sizeof(*out));
    out->n = nc;
    ctx->opt.profile = 0;
    int rc = DGS_OK, best = 0;
    auto render = [&]() {
        return dgs_render(ctx, nodes, n_nodes, env_node_ids, n_envs, max_nodes, node_poses, cams, cams_per_env,
                          max_cams, out_rgb, out_depth, out_alpha, view_pixel_offset, stream_);
    };
    for (int i = 0; i < nc && rc == DGS_OK; ++i) {
        ctx->opt.tile_w = out->tile_w[i] = cand[2 * i];
        ctx->opt.tile_h = out->tile_h[i] = cand[2 * i + 1];
        if ((rc = render())) break;
        cudaEventRecord(a, stream);
        for (int r = 0; r < reps && rc == DGS_OK; ++r) rc = render();
        cudaEventRecord(b, stream);
        cudaEventSynchronize(b);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, a, b);
        out->ms[i] = ms / (float)reps;
        if (out->ms[i] < out->ms[best]) best = i;
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    if (rc != DGS_OK) {
        const std::string why = ctx->err;
        ctx->opt = saved;
        ctx->err = why;
        return rc;
    }
    out->best = best;
    ctx->opt = saved;
    ctx->opt.tile_w = out->tile_w[best];
    ctx->opt.tile_h = out->tile_h[best];
    return render();
}

namespace {

// The adjoint of one view group whose lists are built (K7 then K8).
int enqueue_adjoint(dgs_ctx* ctx, const Batch& B, const GroupLists& G, const float* out_rgb, const float* out_depth,
                    const float* grad_rgb, const float* grad_depth, float* grad_poses, unsigned long long* n_red,
                    cudaStream_t stream, Timer& tm) {
    Launch L{stream, &ctx->launches};
    tm.begin(DGS_K_BACKWARD);
    DGS_CUDA(ctx, cudaMemsetAsync(ctx->inst_grad.p, 0, sizeof(float) * 10 * std::max<uint32_t>(G.n_inst, 1), stream));
    launch_composite_bwd(L, B.d_views, G.v0, G.v1 - G.v0, G.n_tiles, static_cast<uint2*>(G.lb->ranges.p), G.keys, G.vals,
                         static_cast<Record*>(G.lb->records.p), G.P, out_rgb, out_depth, grad_rgb, grad_depth,
                         static_cast<float*>(ctx->inst_grad.p), n_red, G.order, G.ck, G.n_jobs_bound);
    tm.end();
    tm.begin(DGS_K_BACKWARD_PROJECT);
    launch_project_bwd(L, B.dtype_mask, B.d_nodes, B.n_nodes, B.d_views, B.d_vnodes, B.K, B.node_poses,
                       static_cast<InstInfo*>(G.lb->info.p), static_cast<float*>(ctx->inst_grad.p), G.n_inst, G.P,
                       B.d_grads, grad_poses);
    tm.end();
    DGS_CUDA(ctx, cudaGetLastError());
    return DGS_OK;
}

}  // namespace

int dgs_render_backward(dgs_ctx* ctx, const dgs_node* nodes, int32_t n_nodes, const int32_t* env_node_ids,
                        int32_t n_envs, int32_t max_nodes, const float* node_poses, const dgs_camera* cams,
                        const int32_t* cams_per_env, int32_t max_cams, const float* out_rgb, const float* out_depth,
                        const float* grad_rgb, const float* grad_depth, const dgs_node_grads* grads,
                        float* grad_poses, const int64_t* view_pixel_offset, void* stream_) {
    if (!ctx) return DGS_ERR_INVALID_ARG;
    begin_call(ctx);
    if (!grad_rgb) return fail(ctx, DGS_ERR_INVALID_ARG, "grad_rgb is required");
    if (!ctx->aug.empty())
        return fail(ctx, DGS_ERR_UNSUPPORTED, "a randomisation is set: the adjoint needs the un-randomised forward "
                                              "outputs (clear it with dgs_set_augment(ctx, NULL, 0, ...))");
    cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_);
    Timer tm{ctx, stream, ctx->opt.profile != 0};
    int rc;
    unsigned long long* n_red = nullptr;
    // keep_lists: the last render on this context kept the lists of this very batch
    SavedForward* S = ctx->opt.keep_lists && ctx->saved && ctx->saved->valid ? ctx->saved.get() : nullptr;
    if (S && S->sig != call_signature(nodes, n_nodes, env_node_ids, n_envs, max_nodes, node_poses, cams,
                                      cams_per_env, max_cams, view_pixel_offset))
        S = nullptr;
    Batch fresh;
    Batch& B = S ? S->B : fresh;
    if (S) {
        if (!out_rgb || !out_depth) return fail(ctx, DGS_ERR_INVALID_ARG, "out_rgb and out_depth are required");
        ctx->stats = S->stats;
        ctx->stats.path = DGS_PATH_KEPT_LISTS;
        // the gradient table travels through the pinned staging buffer, whose previous upload
        // ended before the previous call returned
        const size_t bytes = sizeof(dgs_node_grads) * (size_t)B.n_nodes;
        char* hm = static_cast<char*>(ctx->h_meta) + (reinterpret_cast<const char*>(B.d_grads) -
                                                      static_cast<const char*>(ctx->meta.p));
        if (grads) std::memcpy(hm, grads, bytes);
        else std::memset(hm, 0, bytes);
        DGS_CUDA(ctx, cudaMemcpyAsync(const_cast<dgs_node_grads*>(B.d_grads), hm, bytes, cudaMemcpyHostToDevice, stream));
        DGS_CUDA(ctx, cudaMemsetAsync(B.d_err, 0, kErrBlockBytes, stream));
    } else {
        rc = prepare(ctx, nodes, n_nodes, env_node_ids, n_envs, max_nodes, node_poses, cams, cams_per_env, max_cams,
                     out_rgb, out_depth, view_pixel_offset, grads, stream, tm, B);
        if (rc != DGS_OK || B.V == 0) return rc;
    }
    uint64_t max_inst = 1;
    if (S)
        for (const GroupLists& G : S->groups) max_inst = std::max<uint64_t>(max_inst, G.n_inst);
    else
        for (auto& g : B.groups) max_inst = std::max<uint64_t>(max_inst, B.inst_at[g.second] - B.inst_at[g.first]);
    if ((rc = ensure(ctx, ctx->inst_grad, sizeof(float) * 10 * max_inst))) return rc;
    if (ctx->opt.profile >= 2) {
        n_red = reinterpret_cast<unsigned long long*>(static_cast<char*>(ctx->errword.p) + 56);
        DGS_CUDA(ctx, cudaMemsetAsync(n_red, 0, sizeof(unsigned long long), stream));
    }
    const int ng = S ? (int)S->groups.size() : (int)B.groups.size();
    for (int g = 0; g < ng; ++g) {
        GroupLists G;
        if (S) G = S->groups[g];
        else build_group_lists(ctx, B, g, ctx->lists[0], stream, tm, G, false);   // no forward: no checkpoints
        if ((rc = enqueue_adjoint(ctx, B, G, out_rgb, out_depth, grad_rgb, grad_depth, grad_poses, n_red, stream, tm)))
            return rc;
    }
    rc = finish(ctx, B, stream);
    if (S) ctx->stats.n_pairs = S->stats.n_pairs;
    if (rc == DGS_OK && n_red) {
        unsigned long long h = 0;
        DGS_CUDA(ctx, cudaMemcpy(&h, n_red, sizeof(h), cudaMemcpyDeviceToHost));
        ctx->stats.bwd_reductions = (int64_t)h;
    }
    return rc;
}

int dgs_pose_twist_grad(const float* poses, const float* grad_poses, int64_t n, float* out_twist, void* stream_) {
    if (n < 0 || (n > 0 && (!poses || !grad_poses || !out_twist))) return DGS_ERR_INVALID_ARG;
    if (n == 0) return DGS_OK;
    int64_t launches = 0;
    launch_pose_twist(Launch{reinterpret_cast<cudaStream_t>(stream_), &launches}, poses, grad_poses, n, out_twist);
    return cudaGetLastError() == cudaSuccess ? DGS_OK : DGS_ERR_CUDA;
}

int dgs_set_augment(dgs_ctx* ctx, const dgs_augment* aug, int32_t n_views, const uint8_t* overlay,
                    int32_t n_frames, int32_t overlay_w, int32_t overlay_h) {
    if (!ctx) return DGS_ERR_INVALID_ARG;
    ctx->err.clear();
    if (n_views < 0) return fail(ctx, DGS_ERR_INVALID_ARG, "n_views must be >= 0");
    if (!aug || n_views == 0) {
        ctx->aug.clear();
        ctx->overlay = nullptr;
        ctx->ov_n = ctx->ov_w = ctx->ov_h = 0;
        return DGS_OK;
    }
    if (overlay && (n_frames < 1 || n_frames > 32768 || overlay_w < 1 || overlay_w > 32768 || overlay_h < 1 ||
                    overlay_h > 32768))
        return fail(ctx, DGS_ERR_INVALID_ARG, "overlay: n_frames, overlay_w and overlay_h must be 1..32768");
    for (int v = 0; v < n_views; ++v) {
        const dgs_augment& a = aug[v];
        const std::string at = "view " + std::to_string(v) + ": ";
        if (!finite(a.hue_shift)) return fail(ctx, DGS_ERR_INVALID_ARG, at + "hue_shift must be finite");
        if (!(a.sat_scale >= 0.f) || !finite(a.sat_scale) || !(a.val_scale >= 0.f) || !finite(a.val_scale))
            return fail(ctx, DGS_ERR_INVALID_ARG, at + "sat_scale and val_scale must be finite and >= 0");
        if (!(a.gamma > 0.f) || !finite(a.gamma)) return fail(ctx, DGS_ERR_INVALID_ARG, at + "gamma must be finite and > 0");
        if (!(a.overlay_beta >= 0.f && a.overlay_beta <= 1.f))
            return fail(ctx, DGS_ERR_INVALID_ARG, at + "overlay_beta must be in [0, 1]");
        if (a.overlay_beta > 0.f) {
            if (!overlay) return fail(ctx, DGS_ERR_INVALID_ARG, at + "overlay_beta > 0 needs an overlay");
            if (a.overlay_frame < 0 || a.overlay_frame >= n_frames || a.overlay_x < 0 || a.overlay_x >= overlay_w ||
                a.overlay_y < 0 || a.overlay_y >= overlay_h)
                return fail(ctx, DGS_ERR_INVALID_ARG, at + "overlay frame or crop origin out of range");
        }
    }
    ctx->aug.assign(aug, aug + n_views);
    ctx->overlay = overlay;
    ctx->ov_n = overlay ? n_frames : 0;
    ctx->ov_w = overlay ? overlay_w : 0;
    ctx->ov_h = overlay ? overlay_h : 0;
    return DGS_OK;
}

int dgs_augment_rgb(dgs_ctx* ctx, float* rgb, const int32_t* view_size, const int64_t* view_pixel_offset,
                    int32_t n_views, void* stream_) {
    if (!ctx) return DGS_ERR_INVALID_ARG;
    begin_call(ctx);
    if (ctx->aug.empty()) return fail(ctx, DGS_ERR_INVALID_ARG, "no randomisation is set (dgs_set_augment)");
    if (n_views != (int64_t)ctx->aug.size())
        return fail(ctx, DGS_ERR_INVALID_ARG, "the randomisation is set for " + std::to_string(ctx->aug.size()) +
                                                  " views, n_views is " + std::to_string(n_views));
    if (!rgb || !view_size) return fail(ctx, DGS_ERR_INVALID_ARG, "rgb and view_size are required");
    const int V = n_views;
    std::vector<AugSpan> spans(V);
    int64_t q = 0, packed = 0;            // quads so far, pixels so far
    for (int v = 0; v < V; ++v) {
        const int32_t w = view_size[2 * v], h = view_size[2 * v + 1];
        if (w < 1 || h < 1 || w > 32768 || h > 32768) return fail(ctx, DGS_ERR_INVALID_ARG, "view size must be 1..32768");
        const int64_t off = view_pixel_offset ? view_pixel_offset[v] : packed;
        if (off < 0) return fail(ctx, DGS_ERR_INVALID_ARG, "negative view_pixel_offset");
        const int64_t n = (int64_t)w * h;
        spans[v] = AugSpan{off, q, w, h};
        q += (off + n - 1) / 4 - off / 4 + 1;    // quads of 4 output pixels holding the view
        packed += n;
    }
    cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_);
    const size_t o_aug = align_up(sizeof(AugSpan) * V, 256);
    const size_t bytes = o_aug + sizeof(dgs_augment) * V;
    // the buffer is read by this pass only, never by a captured graph: its reallocation does
    // not invalidate one
    const uint64_t gen = ctx->gen;
    int rc = ensure(ctx, ctx->aug_dev, bytes);
    ctx->gen = gen;
    if (rc) return rc;
    if ((rc = ensure_host(ctx, ctx->h_aug, ctx->h_aug_bytes, bytes))) return rc;
    if (!ctx->aug_copied) DGS_CUDA(ctx, cudaEventCreateWithFlags(&ctx->aug_copied, cudaEventDisableTiming));
    else DGS_CUDA(ctx, cudaEventSynchronize(ctx->aug_copied));   // the previous upload from the staging is done
    char* hs = static_cast<char*>(ctx->h_aug);
    std::memcpy(hs, spans.data(), sizeof(AugSpan) * V);
    std::memcpy(hs + o_aug, ctx->aug.data(), sizeof(dgs_augment) * V);
    char* ds = static_cast<char*>(ctx->aug_dev.p);
    DGS_CUDA(ctx, cudaMemcpyAsync(ds, hs, bytes, cudaMemcpyHostToDevice, stream));
    DGS_CUDA(ctx, cudaEventRecord(ctx->aug_copied, stream));
    Launch L{stream, &ctx->launches};
    Timer tm{ctx, stream, ctx->opt.profile != 0};
    tm.begin(DGS_K_AUGMENT);
    launch_augment(L, reinterpret_cast<const AugSpan*>(ds), V, q, reinterpret_cast<const dgs_augment*>(ds + o_aug),
                   ctx->overlay, ctx->ov_w, ctx->ov_h, rgb);
    tm.end();
    DGS_CUDA(ctx, cudaGetLastError());
    if (ctx->opt.profile) {
        DGS_CUDA(ctx, cudaStreamSynchronize(stream));
        collect_times(ctx);
    }
    return DGS_OK;
}

}  // extern "C"

// ------------------------------------------------------------------------------------- LiDAR
namespace {


int check_nodes(dgs_ctx* ctx, const dgs_node* nodes, int32_t n_nodes) {
    if (n_nodes < 1 || !nodes) return fail(ctx, DGS_ERR_INVALID_ARG, "nodes: need n_nodes >= 1 and a node array");
    int64_t total = 0;
    for (int k = 0; k < n_nodes; ++k) {
        const dgs_node& nd = nodes[k];
        if (nd.n < 0 || nd.sh_degree < 0 || nd.sh_degree > 3 || nd.dtype < 0 || nd.dtype > 2)
            return fail(ctx, DGS_ERR_INVALID_ARG, "node " + std::to_string(k) + ": bad n, sh_degree or dtype");
        if (nd.n > 0 && (!nd.mean || !nd.log_scale || !nd.quat || !nd.opacity_logit))
            return fail(ctx, DGS_ERR_INVALID_ARG, "node " + std::to_string(k) + ": null attribute pointer");
        total += nd.n;
    }
    if (total >= (1ll << 32)) return fail(ctx, DGS_ERR_INVALID_ARG, "more than 2^32 Gaussians");
    return DGS_OK;
}

}  // namespace

extern "C" {

int dgs_lidar_build(dgs_ctx* ctx, const dgs_node* nodes, int32_t n_nodes, void* stream_) {
    if (!ctx) return DGS_ERR_INVALID_ARG;
    begin_call(ctx);
    int rc = check_nodes(ctx, nodes, n_nodes);
    if (rc) return rc;
    cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_);
    ctx->lid_nodes.clear();
    std::vector<int64_t> P(n_nodes), rec_off(n_nodes), box_off(n_nodes);
    int64_t n_rec = 0, n_box = 0, maxP = 0;
    for (int k = 0; k < n_nodes; ++k) {
        const int64_t nodes2 = (int64_t)lidar_tree_nodes(nodes[k].n);
        P[k] = nodes2 / 2;
        rec_off[k] = n_rec;
        box_off[k] = n_box;
        n_rec += nodes[k].n;
        n_box += nodes2;
        maxP = std::max(maxP, P[k]);
    }
    // level jobs: for h = maxP/2 .. 1, every tree with P >= 2h
    std::vector<std::pair<int64_t, std::vector<std::pair<int, int64_t>>>> levels;
    size_t n_jobs = 0;
    for (int64_t h = maxP / 2; h >= 1; h /= 2) {
        std::vector<std::pair<int, int64_t>> jobs;
        int64_t first = 0;
        for (int k = 0; k < n_nodes; ++k)
            if (P[k] >= 2 * h) { jobs.push_back({k, first}); first += h; }
        n_jobs += jobs.size();
        levels.push_back({h, std::move(jobs)});
    }
    const size_t jb = lidar_level_job_bytes();
    const size_t o_jobs = align_up(sizeof(LidarTreeDev) * n_nodes, 256);
    const size_t tab_bytes = o_jobs + jb * std::max<size_t>(n_jobs, 1);
    if ((rc = ensure(ctx, ctx->lid_rec, sizeof(float4) * 4 * std::max<int64_t>(n_rec, 1)))) return rc;
    if ((rc = ensure(ctx, ctx->lid_box, sizeof(float4) * 2 * std::max<int64_t>(n_box, 1)))) return rc;
    if ((rc = ensure(ctx, ctx->lid_tab, tab_bytes))) return rc;
    float4* rec = static_cast<float4*>(ctx->lid_rec.p);
    float4* box = static_cast<float4*>(ctx->lid_box.p);
    std::vector<char> host(tab_bytes, 0);
    int64_t gbase = 0;
    for (int k = 0; k < n_nodes; ++k) {
        LidarTreeDev t{box + 2 * box_off[k], rec + 4 * rec_off[k], nodes[k].n, P[k], (uint32_t)gbase};
        std::memcpy(host.data() + sizeof(LidarTreeDev) * k, &t, sizeof(t));
        gbase += nodes[k].n;
    }
    size_t ji = 0;
    for (auto& lv : levels)
        for (auto& j : lv.second) lidar_level_job(host.data() + o_jobs, (int)ji++, box + 2 * box_off[j.first], j.second);
    DGS_CUDA(ctx, cudaMemcpyAsync(ctx->lid_tab.p, host.data(), tab_bytes, cudaMemcpyHostToDevice, stream));
    Launch L{stream, &ctx->launches};
    gbase = 0;
    for (int k = 0; k < n_nodes; ++k) {
        NodeDesc nd{};
        nd.mean = nodes[k].mean; nd.log_scale = nodes[k].log_scale; nd.quat = nodes[k].quat;
        nd.opac = nodes[k].opacity_logit; nd.sh = nodes[k].sh; nd.n = nodes[k].n; nd.gbase = gbase;
        nd.deg = nodes[k].sh_degree; nd.dtype = nodes[k].dtype;
        launch_lidar_records(L, nd, ctx->opt.q_max, rec + 4 * rec_off[k], box + 2 * box_off[k], P[k]);
        gbase += nodes[k].n;
    }
    ji = 0;
    for (auto& lv : levels) {
        const int64_t total = lv.first * (int64_t)lv.second.size();
        launch_lidar_level(L, static_cast<char*>(ctx->lid_tab.p) + o_jobs + jb * ji, (int)lv.second.size(), lv.first,
                           total);
        ji += lv.second.size();
    }
    DGS_CUDA(ctx, cudaGetLastError());
    DGS_CUDA(ctx, cudaStreamSynchronize(stream));   // the host table above must outlive its copy
    ctx->lid_nodes.assign(nodes, nodes + n_nodes);
    return DGS_OK;
}

int dgs_lidar_trace(dgs_ctx* ctx, const dgs_node* nodes, int32_t n_nodes, const int32_t* env_node_ids, int32_t n_envs,
                    int32_t max_nodes, const float* node_poses, const dgs_lidar* sensors, int32_t n_sensors,
                    const float* dirs, int32_t n_dirs, float r_min, float r_max, float* out_d, float* out_a,
                    void* stream_) {
    if (!ctx) return DGS_ERR_INVALID_ARG;
    begin_call(ctx);
    int rc = check_nodes(ctx, nodes, n_nodes);
    if (rc) return rc;
    if ((int)ctx->lid_nodes.size() != n_nodes)
        return fail(ctx, DGS_ERR_INVALID_ARG, "no LiDAR structures for these nodes (call dgs_lidar_build)");
    for (int k = 0; k < n_nodes; ++k) {
        const dgs_node &a = nodes[k], &b = ctx->lid_nodes[k];
        if (a.n != b.n || a.mean != b.mean || a.log_scale != b.log_scale || a.quat != b.quat ||
            a.opacity_logit != b.opacity_logit || a.dtype != b.dtype)
            return fail(ctx, DGS_ERR_INVALID_ARG, "node " + std::to_string(k) + " differs from the one built (call dgs_lidar_build)");
    }
    if (n_envs < 1 || max_nodes < 1) return fail(ctx, DGS_ERR_INVALID_ARG, "n_envs and max_nodes must be >= 1");
    if (n_sensors < 0 || n_dirs < 1) return fail(ctx, DGS_ERR_INVALID_ARG, "n_sensors >= 0 and n_dirs >= 1 required");
    if (!env_node_ids || !node_poses || (n_sensors > 0 && (!sensors || !dirs || !out_d || !out_a)))
        return fail(ctx, DGS_ERR_INVALID_ARG, "null pointer argument");
    if (!(r_min >= 0.f) || !(r_max > r_min) || !finite(r_max))
        return fail(ctx, DGS_ERR_INVALID_ARG, "range window: need 0 <= r_min < r_max, finite");
    const int E = n_envs, K = max_nodes;
    std::vector<int> seen(n_nodes, -1);
    for (int e = 0; e < E; ++e)
        for (int j = 0; j < K; ++j) {
            const int k = env_node_ids[(int64_t)e * K + j];
            if (k < -1 || k >= n_nodes) return fail(ctx, DGS_ERR_INVALID_ARG, "env_node_ids out of range");
            if (k >= 0) {
                if (seen[k] == e) return fail(ctx, DGS_ERR_INVALID_ARG, "a node appears twice in one env");
                seen[k] = e;
            }
        }
    std::vector<LidarSensorDev> sd(n_sensors);
    for (int s = 0; s < n_sensors; ++s) {
        const dgs_lidar& L = sensors[s];
        if (L.env < 0 || L.env >= E) return fail(ctx, DGS_ERR_INVALID_ARG, "sensor env out of range");
        for (int a = 0; a < 12; ++a)
            if (!finite(L.world_from_sensor[a])) return fail(ctx, DGS_ERR_INVALID_ARG, "sensor pose not finite");
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) {
                double d = 0;
                for (int r = 0; r < 3; ++r) d += (double)L.world_from_sensor[r * 4 + a] * L.world_from_sensor[r * 4 + b];
                if (std::fabs(d - (a == b ? 1.0 : 0.0)) > 1e-4)
                    return fail(ctx, DGS_ERR_INVALID_ARG, "sensor rotation not orthonormal");
            }
        sd[s].env = L.env;
        std::memcpy(sd[s].pose, L.world_from_sensor, sizeof(sd[s].pose));
    }
    if (n_sensors == 0) return DGS_OK;
    cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_);
    const size_t o_slot = align_up(sizeof(LidarSensorDev) * n_sensors, 256);
    const size_t bytes = o_slot + sizeof(int32_t) * (size_t)E * K;
    if ((rc = ensure(ctx, ctx->lid_meta, bytes))) return rc;
    if ((rc = ensure(ctx, ctx->lid_slots, sizeof(LidarSlot) * (size_t)n_sensors * K))) return rc;
    if ((rc = ensure(ctx, ctx->errword, 64))) return rc;
    if ((rc = ensure_host(ctx, ctx->h_lid, ctx->h_lid_bytes, bytes))) return rc;
    DGS_CUDA(ctx, cudaStreamSynchronize(stream));   // the previous call's upload from the staging
    char* h = static_cast<char*>(ctx->h_lid);
    std::memcpy(h, sd.data(), sizeof(LidarSensorDev) * n_sensors);
    std::memcpy(h + o_slot, env_node_ids, sizeof(int32_t) * (size_t)E * K);
    char* d = static_cast<char*>(ctx->lid_meta.p);
    uint32_t* err = static_cast<uint32_t*>(ctx->errword.p);
    DGS_CUDA(ctx, cudaMemsetAsync(err, 0, 64, stream));
    DGS_CUDA(ctx, cudaMemcpyAsync(d, h, bytes, cudaMemcpyHostToDevice, stream));
    Launch L{stream, &ctx->launches};
    Timer tm{ctx, stream, ctx->opt.profile != 0};
    tm.begin(DGS_K_LIDAR);
    LidarSlot* slots = static_cast<LidarSlot*>(ctx->lid_slots.p);
    launch_lidar_setup(L, reinterpret_cast<const LidarSensorDev*>(d), n_sensors,
                       reinterpret_cast<const int32_t*>(d + o_slot), K, node_poses, slots, err);
    LidarParams LP{r_min, r_max, ctx->opt.alpha_min, ctx->opt.alpha_max, ctx->opt.t_min, ctx->opt.q_max};
    launch_lidar_trace(L, static_cast<const LidarTreeDev*>(ctx->lid_tab.p), slots, K, dirs, n_dirs,
                       (int64_t)n_sensors * n_dirs, LP, out_d, out_a, err,
                       reinterpret_cast<unsigned long long*>(static_cast<char*>(ctx->errword.p) + 8));
    tm.end();
    DGS_CUDA(ctx, cudaGetLastError());
    uint32_t errw = 0;
    DGS_CUDA(ctx, cudaMemcpyAsync(&errw, err, sizeof(uint32_t), cudaMemcpyDeviceToHost, stream));
    DGS_CUDA(ctx, cudaStreamSynchronize(stream));
    collect_times(ctx);
    if (errw & kErrPose) return fail(ctx, DGS_ERR_INVALID_ARG, "a node pose is not finite or not rigid");
    if (errw & kErrCapacity) return fail(ctx, DGS_ERR_CUDA, "internal: BVH traversal stack overflow");
    return DGS_OK;
}

}  // extern "C"

extern "C" {

int dgs_mesh_to_gaussians(dgs_ctx* ctx, const float* vertices, int64_t n_vertices, const int32_t* faces,
                          int64_t n_faces, const float* vertex_colors, float flatten, float opacity_logit,
                          int32_t sh_degree, float* out_mean, float* out_log_scale, float* out_quat,
                          float* out_opacity_logit, float* out_sh, void* stream_) {
    if (!ctx) return DGS_ERR_INVALID_ARG;
    begin_call(ctx);
    if (n_faces < 0 || n_vertices < 0 || n_vertices >= (1ll << 31))
        return fail(ctx, DGS_ERR_INVALID_ARG, "need n_faces >= 0 and 0 <= n_vertices < 2^31");
    if (!(flatten > 0.f && flatten <= 1.f)) return fail(ctx, DGS_ERR_INVALID_ARG, "flatten must be in (0, 1]");
    if (!finite(opacity_logit)) return fail(ctx, DGS_ERR_INVALID_ARG, "opacity_logit must be finite");
    if (sh_degree < 0 || sh_degree > 3) return fail(ctx, DGS_ERR_INVALID_ARG, "sh_degree must be 0..3");
    if (n_faces == 0) return DGS_OK;
    if (!vertices || !faces || !out_mean || !out_log_scale || !out_quat || !out_opacity_logit || !out_sh)
        return fail(ctx, DGS_ERR_INVALID_ARG, "null pointer argument");
    if (reinterpret_cast<uintptr_t>(out_quat) % 16) return fail(ctx, DGS_ERR_INVALID_ARG, "out_quat must be 16-byte aligned");
    cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_);
    int rc;
    if ((rc = ensure(ctx, ctx->errword, 64))) return rc;
    uint32_t* err = static_cast<uint32_t*>(ctx->errword.p);
    DGS_CUDA(ctx, cudaMemsetAsync(err, 0, 64, stream));
    Launch L{stream, &ctx->launches};
    Timer tm{ctx, stream, ctx->opt.profile != 0};
    tm.begin(DGS_K_MESH);
    launch_mesh_gaussians(L, vertices, n_vertices, faces, n_faces, vertex_colors, flatten, opacity_logit,
                          (sh_degree + 1) * (sh_degree + 1), out_mean, out_log_scale, out_quat, out_opacity_logit, out_sh,
                          err);
    tm.end();
    DGS_CUDA(ctx, cudaGetLastError());
    uint32_t errw = 0;
    DGS_CUDA(ctx, cudaMemcpyAsync(&errw, err, sizeof(uint32_t), cudaMemcpyDeviceToHost, stream));
    DGS_CUDA(ctx, cudaStreamSynchronize(stream));
    collect_times(ctx);
    if (errw & kErrIndex) return fail(ctx, DGS_ERR_INVALID_ARG, "a face index is outside [0, n_vertices)");
    return DGS_OK;
}

}  // extern "C"

extern "C" {

int dgs_tsdf_integrate(dgs_ctx* ctx, float* tsdf, float* weight, int32_t nx, int32_t ny, int32_t nz,
                       const float* origin, float voxel, float trunc, float max_weight, float min_alpha,
                       const dgs_camera* cams, int32_t n_views, const float* depth, const float* alpha,
                       const int64_t* view_pixel_offset, void* stream_) {
    if (!ctx) return DGS_ERR_INVALID_ARG;
    begin_call(ctx);
    if (nx < 1 || ny < 1 || nz < 1 || (int64_t)nx * ny * nz >= (1ll << 31))
        return fail(ctx, DGS_ERR_INVALID_ARG, "grid: need nx, ny, nz >= 1 and nx*ny*nz < 2^31");
    if (!origin || !finite(origin[0]) || !finite(origin[1]) || !finite(origin[2]))
        return fail(ctx, DGS_ERR_INVALID_ARG, "origin must be 3 finite values");
    if (!(voxel > 0.f) || !finite(voxel) || !(trunc > 0.f) || !finite(trunc) || !(max_weight > 0.f) ||
        !finite(max_weight) || !(min_alpha > 0.f && min_alpha <= 1.f))
        return fail(ctx, DGS_ERR_INVALID_ARG, "need voxel, trunc, max_weight > 0 (finite) and min_alpha in (0, 1]");
    if (n_views < 0) return fail(ctx, DGS_ERR_INVALID_ARG, "n_views must be >= 0");
    if (!tsdf || !weight || (n_views > 0 && (!cams || !depth || !alpha)))
        return fail(ctx, DGS_ERR_INVALID_ARG, "null pointer argument");
    if (n_views == 0) return DGS_OK;
    std::vector<TsdfView> views(n_views);
    int64_t packed = 0;
    for (int v = 0; v < n_views; ++v) {
        const dgs_camera& c = cams[v];
        if (c.width < 1 || c.height < 1 || c.width > 32768 || c.height > 32768)
            return fail(ctx, DGS_ERR_INVALID_ARG, "camera resolution");
        if (!(c.fx > 0) || !(c.fy > 0) || !finite(c.fx) || !finite(c.fy) || !finite(c.cx) || !finite(c.cy))
            return fail(ctx, DGS_ERR_INVALID_ARG, "camera intrinsics");
        for (int a = 0; a < 12; ++a)
            if (!finite(c.cam_from_world[a])) return fail(ctx, DGS_ERR_INVALID_ARG, "camera pose not finite");
        TsdfView& tv = views[v];
        for (int a = 0; a < 3; ++a) {
            for (int b = 0; b < 3; ++b) tv.R[3 * a + b] = c.cam_from_world[4 * a + b];
            tv.t[a] = c.cam_from_world[4 * a + 3];
        }
        tv.fx = c.fx; tv.fy = c.fy; tv.cx = c.cx; tv.cy = c.cy; tv.W = c.width; tv.H = c.height;
        tv.pix_off = view_pixel_offset ? view_pixel_offset[v] : packed;
        if (tv.pix_off < 0) return fail(ctx, DGS_ERR_INVALID_ARG, "negative view_pixel_offset");
        tv.q0 = packed;
        packed += (int64_t)c.width * c.height;
    }
    cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_);
    const size_t bytes = sizeof(TsdfView) * n_views;
    const uint64_t gen = ctx->gen;               // read by this call only, never by a captured graph
    int rc = ensure(ctx, ctx->tsdf_meta, bytes);
    if (!rc) rc = ensure(ctx, ctx->tsdf_depth, sizeof(float) * packed);
    ctx->gen = gen;
    if (rc) return rc;
    if ((rc = ensure_host(ctx, ctx->h_tsdf, ctx->h_tsdf_bytes, bytes))) return rc;
    if (!ctx->tsdf_copied) DGS_CUDA(ctx, cudaEventCreateWithFlags(&ctx->tsdf_copied, cudaEventDisableTiming));
    else DGS_CUDA(ctx, cudaEventSynchronize(ctx->tsdf_copied));
    std::memcpy(ctx->h_tsdf, views.data(), bytes);
    DGS_CUDA(ctx, cudaMemcpyAsync(ctx->tsdf_meta.p, ctx->h_tsdf, bytes, cudaMemcpyHostToDevice, stream));
    DGS_CUDA(ctx, cudaEventRecord(ctx->tsdf_copied, stream));
    TsdfParams TP{origin[0], origin[1], origin[2], voxel, trunc, 1.f / trunc, max_weight, min_alpha};
    Launch L{stream, &ctx->launches};
    Timer tm{ctx, stream, ctx->opt.profile != 0};
    tm.begin(DGS_K_TSDF);
    launch_tsdf(L, tsdf, weight, nx, ny, (int64_t)nx * ny * nz, TP, static_cast<const TsdfView*>(ctx->tsdf_meta.p),
                n_views, depth, alpha, static_cast<float*>(ctx->tsdf_depth.p), packed);
    tm.end();
    DGS_CUDA(ctx, cudaGetLastError());
    if (ctx->opt.profile) {
        DGS_CUDA(ctx, cudaStreamSynchronize(stream));
        collect_times(ctx);
    }
    return DGS_OK;
}

}  // extern "C"
