// Internal device structures and helpers of libdgs (sm_103a): the splatting renderer of
// Sec. III-A / III-C and the side workloads of Sec. III-B, III-C and IV share them.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "dgs.h"

namespace dgs {

constexpr int kWarp = 32;
constexpr int kChunk = 32;           // Gaussians per chunk: one warp projects one chunk
constexpr int kZBits = 28;           // bits of the depth field of a sort key
constexpr uint32_t kMaxPairs = (1u << 30) - 1;   // per view group (30-bit scan counters)
// Tile keys of the (tile, instance) pairs: bits 0..23 the view within the view group above the
// tile's index within its view (Params::tbits bits), bits 24..31 the mask of the tile's
// 8x4-pixel sub-tiles that the instance's ellipse reaches (bit s = sub-tile (s mod (tile_w/8),
// s div (tile_w/8))).  The instances are sorted by view, then depth, so each instance's pairs
// come out view by view; the tile sort then radixes the tbits bits only, and a tile's run is
// in depth order.
constexpr int kTileBits = 24;
constexpr uint32_t kTileMask = (1u << kTileBits) - 1u;
constexpr int64_t kMaxGroupTiles = (1ll << kTileBits) - 1;   // a view group's tiles (the dead key sorts last)

// Device error word bits (ctx status).
constexpr uint32_t kErrPose = 1u;       // non-finite or non-rigid node pose
constexpr uint32_t kErrTimeout = 2u;    // a bounded spin gave up
constexpr uint32_t kErrCapacity = 4u;   // a count exceeded its buffer
constexpr uint32_t kErrMismatch = 8u;   // count and emit passes disagreed on a chunk
constexpr uint32_t kErrIndex = 16u;     // an input index out of range (mesh faces)
constexpr uint32_t kErrBounds = 32u;    // debug builds: a checked index fell outside its bound

// Error block of a call: word 0 the bits above, words 2..15 counters, words 16..21 the first
// failed bounds check (site, unused, index as u64, bound as u64).
constexpr int kErrBlockBytes = 128;
constexpr int kDbgWord = 16;

// Debug builds (compiled with -DDGS_DEBUG).  The kernels of the render and its adjoint check
// every index they take from another kernel's output -- record numbers from the scans, the
// depth-sorted instance numbers, sort scatter destinations, tile-list entries, Gaussian ids --
// against the bound of what it indexes, before the access.  A failed check skips the access,
// sets kErrBounds and records the first failing site, index and bound; the call then returns
// DGS_ERR_CUDA naming the site.  Release builds compile the checks out.
#ifdef DGS_DEBUG
constexpr bool kDebugChecks = true;
#else
constexpr bool kDebugChecks = false;
#endif
enum DbgSite : uint32_t {
    kSiteEmitRecord = 1,      // emission: record number of a visible instance
    kSiteScanInstance,        // tile-count scan: depth-sorted instance number
    kSitePairsInstance,       // pair writer: depth-sorted instance number
    kSiteSortScatter,         // radix sort: destination of a live key
    kSiteCompositeRecord,     // compositor: instance number of a tile-list entry
    kSiteBackwardRecord,      // adjoint compositor: instance number of a tile-list entry
    kSiteProjectBwdGaussian,  // projection adjoint: Gaussian of an instance within its node
    kSiteCount
};

struct NodeDesc {
    const float* mean;
    const void* log_scale;
    const void* quat;
    const float* opac;
    const void* sh;
    int64_t n;
    int64_t gbase;        // global id of the node's first Gaussian
    int32_t deg;
    int32_t dtype;
    int32_t chunk0;       // first chunk of the node in the node-major chunk numbering
    int32_t nchunks;
};

struct ViewDesc {
    float fx, fy, cx, cy;
    float limx, limy;     // Jacobian clamp of tx/tz and ty/tz
    int32_t W, H;
    int32_t tiles_x, tiles_y;
    int32_t env;
    int32_t tile_base;    // first global tile of the view within its group
    int64_t pix_off;      // first output pixel
    float cam[12];        // cam_from_world
};

// Per (view, slot): the node and its camera_from_node transform.
struct VNode {
    float M[12];          // camera_from_node, row-major 3x4 (leading parts)
    float Ml[12];         // trailing parts: camera_from_node = M + Ml to about 2^-48
    float o[3];           // camera centre in the node frame
    int32_t node;         // -1 = empty slot
    int64_t tab;          // count-table index of the node's first chunk in this view
};

// Error-free transformations in binary32 (Knuth's TwoSum; TwoProduct by a fused multiply-add):
// a + b = s + e and a * b = p + e exactly, barring overflow and underflow.  The _rn intrinsics
// keep the compiler from contracting or reassociating them.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
__device__ __forceinline__ void two_prod(float a, float b, float& p, float& e) {
    p = __fmul_rn(a, b);
    e = __fmaf_rn(a, b, -p);
}

// Row r of camera_from_node applied to a node-frame point, faithfully rounded.  With the row
// held as M + Ml, the products M_j m_j and the sums are carried as unevaluated (value, error)
// pairs (the compensated dot product of Ogita, Rump and Oishi, 2005); the Ml terms, of relative
// size 2^-24, enter the error sum directly.  The result differs from the exact value for the
// FP32 inputs by at most 2^-24 |result| plus terms of order 2^-48 times the magnitude of the
// summands: within one unit in the last place, whatever the scene.
__device__ __forceinline__ float camera_row(const VNode& vn, int r, float mx, float my, float mz) {
    const float* M = vn.M + 4 * r;
    const float* L = vn.Ml + 4 * r;
    float p, s, h, e, q;
    two_prod(M[0], mx, p, s);
    two_prod(M[1], my, h, e);
    two_sum(p, h, p, q);
    s = __fadd_rn(s, __fadd_rn(q, e));
    two_prod(M[2], mz, h, e);
    two_sum(p, h, p, q);
    s = __fadd_rn(s, __fadd_rn(q, e));
    two_sum(p, M[3], p, q);
    s = __fadd_rn(s, q);
    s = __fmaf_rn(L[0], mx, s);
    s = __fmaf_rn(L[1], my, s);
    s = __fmaf_rn(L[2], mz, s);
    s = __fadd_rn(s, L[3]);
    return __fadd_rn(p, s);
}

// Sec. III-A (depth sorting): the depth key is the camera-space z, faithfully rounded.
__device__ __forceinline__ float camera_depth(const VNode& vn, float mx, float my, float mz) {
    return camera_row(vn, 2, mx, my, mz);
}

struct Params {
    float z_near, lowpass, alpha_min, alpha_max, t_min, q_max, guard;
    float bg0, bg1, bg2;
    float qbin;           // binning limit on d^T conic d (q_max with an FP32 safety margin)
    int32_t tile_w, tile_h;
    int32_t tile_sx, tile_sy; // log2 of tile_w, tile_h (valid tile shapes are powers of two)
    int32_t exact_tile_test;
    uint32_t zbase;       // float bits of 2^floor(log2 z_near)
    int32_t tile0;        // first global tile of the current view group
    uint32_t* err;        // device error word
    const uint32_t* gate; // emission is skipped when non-null and *gate != 0 (capacity overflow)
    float p_min;          // kHalfLog2e * q_max: exponents below it are outside the 3-sigma ellipse
    float log2_amin;      // log2(alpha_min) (-inf for alpha_min = 0)
    uint32_t n_rec;       // records of the current view group (bound of its instance numbers)
    uint32_t view0;       // first view of the current view group
    int32_t tbits;        // bits of a tile within its view (tile keys: view in group << tbits | tile)
    int32_t vshift;       // > 0: emission writes instance numbers as r | view in group << vshift
    const uint32_t* inst_base_dev;  // emission: first record of the group read on the device (graph replay)
    // image randomisation of the RGB output (null aug = none): per-view records, overlay clip
    const dgs_augment* aug;
    const uint8_t* overlay;
    int32_t ov_w, ov_h;
};

// Projected instance as stored for compositing: 48 bytes.
//   r0 = (u, v, opacity, z), r1 = (qa, qb, qc, box x), r2 = (r, g, b, box y), with
//   d^T conic d = qa (dx + qb dy)^2 + qc dy^2 and box x/y = pixel index range of the ellipse's
//   bounding box packed as lo | hi << 16.
struct Record {
    float4 r0, r1, r2;
};

// Identity of a projected instance (read by the adjoint): global Gaussian id and the
// (view * K + slot) index of its VNode.
struct InstInfo {
    uint32_t gid;
    uint32_t view;
};

// (view, slot) entries of node k: node_views[node_view_off[k] .. node_view_off[k+1])
struct NodeView {
    int32_t view;
    int32_t slot;
    int64_t tab;          // count-table index of the node's first chunk in this view
};

// Host side of one batch, shared by every entry point that renders: the validated arguments
// as the tables the kernels read.  View v enumerates (env, camera) env-major; the count table
// lists, per view, the 32-Gaussian chunks of its nodes in node-id order.
struct HostTables {
    std::vector<NodeDesc> nodes;
    std::vector<ViewDesc> views;
    std::vector<int> view_env, view_cam;
    std::vector<int32_t> slot_node;    // [V*K] node drawn in slot j of view v's env (-1 = empty)
    std::vector<int64_t> vnode_tab;    // [V*K] count-table entry of (view, slot)'s first chunk
    std::vector<int64_t> view_tab;     // [V+1] first count-table entry of each view; [V] = T
    std::vector<int32_t> pmap;         // [V*(2K+1)] plain mode: per view, chunk prefix and slot of
                                       // each present node in node-id order
    std::vector<int32_t> nv_off;       // [n_nodes+1] node -> its (view, slot) entries in nv
    std::vector<NodeView> nv;
    int dtype_mask = 0;                // storage types present (bit = dgs_dtype)
    int64_t chunk_total = 0, tiles_total = 0, pix_total = 0, n_instances = 0;
    int64_t T = 0;                     // count-table entries
};

// Validates options (0 = invalid, with the reason in `why`).
int check_options(const dgs_options* o, std::string& why);

// Kernel parameters from options (no group offset, error word or randomisation set).
Params make_params(const dgs_options& o);

// Validates a render call's arguments (everything that can be checked on the host: shapes, node
// ids, camera intrinsics and extrinsics, pixel offsets) and builds its HostTables.  Returns
// DGS_OK or the status to report, with the reason in `why`.  Makes no CUDA call.
int build_host_tables(const dgs_options& o, const dgs_node* nodes, int32_t n_nodes, const int32_t* env_node_ids,
                      int32_t n_envs, int32_t max_nodes, const float* node_poses, const dgs_camera* cams,
                      const int32_t* cams_per_env, int32_t max_cams, const int64_t* view_pixel_offset, HostTables& H,
                      std::string& why);

template <int DT>
__device__ __forceinline__ float ld_attr(const void* p, int64_t i) {
    if constexpr (DT == DGS_F32) return __ldg(reinterpret_cast<const float*>(p) + i);
    else if constexpr (DT == DGS_BF16) return __bfloat162float(reinterpret_cast<const __nv_bfloat16*>(p)[i]);
    else return __half2float(reinterpret_cast<const __half*>(p)[i]);
}

__device__ __forceinline__ uint32_t lane_id() { return threadIdx.x & 31u; }

// Flattened warp walk over the units of up to 32 items.  Items are dense (lane k of the warp
// holds item k for k < n_items) and my_excl is item lane's exclusive prefix of unit counts (>= 1
// each).  For the 32 units of a flush starting at `base`, the owner of unit base + lane is the
// last item whose prefix is <= base + lane: the items at or before `base` (one ballot) plus
// those starting inside the flush up to the unit (one OR-reduction of start bits).
__device__ __forceinline__ int walk_owner_of(int lane, bool item, uint32_t my_excl, uint32_t base) {
    const int first = __popc(__ballot_sync(0xffffffffu, item && my_excl <= base)) - 1;
    const uint32_t d = my_excl - base;
    const uint32_t starts = __reduce_or_sync(0xffffffffu, (item && my_excl > base && d < 32u) ? (1u << d) : 0u);
    return first + __popc(starts & ((2u << lane) - 1u));
}

// Compositing arithmetic shared by the forward pass and its adjoint, so both take the same
// FP32 decisions.  exp(-q/2) = 2^(c q) with c = -log2(e)/2: a staged record carries
// (c qa, qb, c qc), each coefficient one FP32 product, and the pixel's exponent is
// p = (c qa) (dx + qb dy)^2 + (c qc) dy^2; the 3-sigma test q <= q_max reads p >= c q_max.
constexpr float kHalfLog2e = -0.72134752044448170f;   // -log2(e) / 2

__device__ __forceinline__ float fast_exp2(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ float fast_log2(float x) {
    float y;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Sec. III-A cutoffs of a record at a pixel, as one threshold on the exponent p (alpha =
// min(alpha_max, o 2^p)): the pixel is skipped unless p >= max(p_min, log2(alpha_min) - log2 o),
// i.e. unless it lies inside the 3-sigma ellipse and its alpha reaches alpha_min.  Taken in the
// log domain, the alpha_min decision moves by about 8 units of 2^-24 relative in alpha (the
// rounding of p and of the two logarithms), inside the FP32 band of that decision; the
// compositor and its adjoint both use this function, so they decide alike.
__device__ __forceinline__ float reach_threshold(const Params& P, float opacity) {
    return fmaxf(P.p_min, P.log2_amin - fast_log2(opacity));
}

// Image randomisation of one pixel (Sec. IV): clamp to [0, 1], linear blend with the overlay
// pixel o (3 bytes; read only when overlay_beta != 0), hue shift and saturation/value scaling
// in the hexcone HSV model, then the power curve c^gamma evaluated as 2^(gamma log2 c).
// Every multiply-add is an explicit fmaf, so the fused and the separate kernel round
// identically.  The hue's sector is chosen with selects, not branches.  HSV -> RGB uses the
// per-channel form c_n = V - V S clamp(min(k, 4 - k), 0, 1), k = (n + 6H) mod 6, n = 5, 3, 1
// for red, green, blue, which equals the six-sector table of the model.
__device__ __forceinline__ void augment_pixel(const dgs_augment& a, const uint8_t* __restrict__ o, float& r,
                                              float& g, float& b) {
    r = fminf(fmaxf(r, 0.f), 1.f);
    g = fminf(fmaxf(g, 0.f), 1.f);
    b = fminf(fmaxf(b, 0.f), 1.f);
    const float beta = a.overlay_beta;
    if (beta != 0.f) {
        constexpr float k255 = 1.f / 255.f;
        r = fmaf(beta, fmaf((float)o[0], k255, -r), r);
        g = fmaf(beta, fmaf((float)o[1], k255, -g), g);
        b = fmaf(beta, fmaf((float)o[2], k255, -b), b);
    }
    const float v = fmaxf(fmaxf(r, g), b), m = fminf(fminf(r, g), b), c = v - m;
    // hue in sixths of a turn from the sector of the largest channel (red first, then green);
    // a chroma <= 1e-30 counts as grey (H = S = 0), which keeps 1/c finite
    const bool grey = !(c > 1e-30f), is_r = v == r, is_g = v == g;
    const float num = is_r ? g - b : (is_g ? b - r : r - g);
    const float off = is_r ? 0.f : (is_g ? 2.f : 4.f);
    float h = grey ? 0.f : __fdividef(num, c) + off;
    if (h < 0.f) h += 6.f;
    const float s = grey ? 0.f : __fdividef(c, v);
    h = fmaf(6.f, a.hue_shift, h);
    h = fmaf(-6.f, floorf(h * (1.f / 6.f)), h);      // [0, 6) up to one rounding
    const float vv = fminf(1.f, v * a.val_scale);
    const float vs = vv * fminf(1.f, s * a.sat_scale);
    float k;
    k = 5.f + h; if (k >= 6.f) k -= 6.f;
    r = fmaf(-vs, fminf(fmaxf(fminf(k, 4.f - k), 0.f), 1.f), vv);
    k = 3.f + h; if (k >= 6.f) k -= 6.f;
    g = fmaf(-vs, fminf(fmaxf(fminf(k, 4.f - k), 0.f), 1.f), vv);
    k = 1.f + h; if (k >= 6.f) k -= 6.f;
    b = fmaf(-vs, fminf(fmaxf(fminf(k, 4.f - k), 0.f), 1.f), vv);
    if (a.gamma != 1.f) {
        r = fast_exp2(a.gamma * fast_log2(r));
        g = fast_exp2(a.gamma * fast_log2(g));
        b = fast_exp2(a.gamma * fast_log2(b));
    }
}

// The overlay pixel a view's pixel (x, y) blends with: frame overlay_frame, row
// (overlay_y + y) mod oh, column (overlay_x + x) mod ow of the [frames, oh, ow, 3] clip.
__device__ __forceinline__ const uint8_t* overlay_pixel(const uint8_t* overlay, int ow, int oh, const dgs_augment& a,
                                                        int x, int y) {
    const int ox = (a.overlay_x + x) % ow, oy = (a.overlay_y + y) % oh;
    return overlay + (((int64_t)a.overlay_frame * oh + oy) * ow + ox) * 3;
}

// Sec. III-A (the splat's falloff at a pixel).  Exponent p of a staged record (scaled
// coefficients ca, qb, cc) at pixel offset (dx, dy);
// also returns t = dx + qb dy.
__device__ __forceinline__ float pixel_exponent(float ca, float qb, float cc, float dx, float dy, float& t) {
    t = fmaf(qb, dy, dx);
    return fmaf(ca * t, t, cc * dy * dy);
}

// Sec. III-A (tile binning at the compositor's granularity).  The ellipse {q <= qlim},
// q = qa (dx + qb dy)^2 + qc dy^2, spans dy in [-ye, ye], ye = sqrt(qlim / qc); at a given dy its
// x-section is -qb dy -+ sqrt((qlim - qc dy^2) / qa).  Its leftmost point lies at
// dy_L = qb sqrt(qa qlim / (qc (qc + qa qb^2))) and its rightmost at -dy_L.  Per-instance
// constants of the sub-tile test: (ye, dy_L, 1/qa).
// (The sub-tile test is a filter with the binning limit's margin of 0.1 % + 1e-3 on q: the
// hardware's approximate square root and division, within a few units of 2^-23, are ample.)
__device__ __forceinline__ float approx_sqrt(float x) {
    float y;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ float4 ellipse_extent(float qa, float qb, float qc, float qlim) {
    const float ye = approx_sqrt(__fdividef(qlim, qc));
    const float dyl = qb * approx_sqrt(__fdividef(qa * qlim, qc * fmaf(qa * qb, qb, qc)));
    return make_float4(ye, dyl, __fdividef(1.f, qa), 0.f);
}

// The ellipse's x-extent over the band of pixel-centre rows [yc0, yc1] (absolute): the part of
// the ellipse in the band is convex, so it is one interval [L, R] of absolute x, with L at the
// clamp of dy_L into the band and R at the clamp of -dy_L (the lower boundary is convex and the
// upper concave in dy).  False if the band misses the ellipse's y-extent.
__device__ __forceinline__ bool band_interval(float u, float v, float qb, float qc, const float4& ext, float yc0,
                                              float yc1, float qlim, float& L, float& R) {
    const float Y0 = fmaxf(yc0 - v, -ext.x), Y1 = fminf(yc1 - v, ext.x);
    if (!(Y0 <= Y1)) return false;
    const float dl = fminf(Y1, fmaxf(Y0, ext.y)), dr = fminf(Y1, fmaxf(Y0, -ext.y));
    L = u + fmaf(-qb, dl, -approx_sqrt(fmaxf(0.f, fmaf(-qc * dl, dl, qlim)) * ext.z));
    R = u + fmaf(-qb, dr, approx_sqrt(fmaxf(0.f, fmaf(-qc * dr, dr, qlim)) * ext.z));
    return true;
}

// Sec. III-A (tile binning).  The tiles of tile row ty that an instance reaches: those whose
// pixel-centre rectangle (clipped to the instance's pixel box [x0, x1] x [y0, y1]) meets the
// ellipse {q <= qbin}.  Within the tile row's band of pixel-centre rows the ellipse's x-extent is
// one interval [L, R] (band_interval), clipped to the box's centres; tile t's centres span
// [t w + 1/2, t w + w - 1/2], so the tiles reached are the run t0 = ceil((L + 1/2) / w) - 1 ..
// t1 = floor((R - 1/2) / w) (w a power of two: the divisions are exact).  Without the exact
// test, every tile the box row covers.  Returns the run's length (0: none) and t0.  The emission
// count and the pair writer call this on the same stored record values, so they agree exactly.
__device__ __forceinline__ int tile_row_run(float u, float v, float qb, float qc, const float4& ext, int x0, int x1,
                                            int y0, int y1, int ty, const Params& P, int& t0) {
    const int py0 = max(ty * P.tile_h, y0), py1 = min(ty * P.tile_h + P.tile_h - 1, y1);
    if (py0 > py1) return 0;
    float L = (float)x0 + 0.5f, R = (float)x1 + 0.5f;
    if (P.exact_tile_test) {
        float l, r;
        if (!band_interval(u, v, qb, qc, ext, (float)py0 + 0.5f, (float)py1 + 0.5f, P.qbin, l, r)) return 0;
        L = fmaxf(L, l);
        R = fminf(R, r);
        if (!(L <= R)) return 0;
    }
    const float iw = 1.f / (float)P.tile_w;
    t0 = (int)ceilf((L + 0.5f) * iw) - 1;
    const int t1 = (int)floorf((R - 0.5f) * iw);
    return max(0, t1 - t0 + 1);
}

__device__ __forceinline__ uint64_t global_timer_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// ------------------------------------------------------------------ launchers (host side)
struct Launch {
    cudaStream_t stream;
    int64_t* launches;    // incremented per kernel launch
};

void launch_setup_views(const Launch& L, const ViewDesc* views, int n_views, const float* node_poses,
                        const int32_t* view_slots_node, int K, VNode* vnodes, const int64_t* vnode_tab,
                        uint32_t* err);

void launch_count(const Launch& L, int dtype_mask, const NodeDesc* nodes, int n_nodes, const ViewDesc* views,
                  const VNode* vnodes, int K, const NodeView* node_views, const int32_t* node_view_off,
                  int n_chunks_total, const Params& P, int v0, int v1, bool batched, const int32_t* view_chunk_nodes,
                  int64_t view_chunks, uint2* counts);

void launch_scan(const Launch& L, const uint2* counts, int64_t n, uint32_t* inst_off, uint64_t* pair_off,
                 ulonglong2* parts, int64_t n_parts_cap);

// K2: for every visible instance of views [v0, v1): its record, identity, depth key
// (bits(z32) - zbase saturated to 28 bits), its own index (the value the depth sort carries)
// and its number of tile pairs, at the scanned instance offsets minus inst_base.
void launch_emit(const Launch& L, int dtype_mask, const NodeDesc* nodes, int n_nodes, const ViewDesc* views,
                 const VNode* vnodes, int K, const NodeView* node_views, const int32_t* node_view_off,
                 int n_chunks_total, const Params& P, int v0, int v1, bool batched, const int32_t* view_chunk_nodes,
                 int64_t view_chunks, const uint2* counts, const uint32_t* inst_off, uint32_t inst_base,
                 Record* records, InstInfo* info, uint32_t* dkey, uint32_t* ival, uint32_t* ntile, uint32_t* vig);

// Bounded waits of the sort: the look-back spin limit, and a test of it (mute_part: the
// partition of the first digit pass that publishes no status; ~0 = none).
struct SortCtl {
    uint64_t spin_ns = 1000000000ull;
    uint32_t mute_part = 0xFFFFFFFFu;
    bool runs = false;    // neighbouring keys share their high digits (histogram by runs)
};

// The depth sort's most significant key: the view of each instance within its view group.
// The instance numbers of a group are emitted view by view, view j of the group holding
// inst_off[view_tab[v0 + j + 1]] - inst_off[view_tab[v0 + j]] of them (the count scan), which
// gives the view key's histogram.  With vshift > 0 the values are packed, r | view << vshift
// (r < 2^vshift), and the last view pass leaves r; else the view of value r is vig[r].
struct ViewKey {
    int bits = 0;                        // view bits; 0: no view passes
    int vshift = 0;
    const uint32_t* vig = nullptr;
    const uint32_t* inst_off = nullptr;  // count-scan offsets (device)
    const int64_t* view_tab = nullptr;   // first count-table entry of each view (device)
    int v0 = 0, nv = 0;
};

// Stable LSD radix sort of (key, value) on the low key_bits bits.  With d_n non-null the
// number of pairs is read on the device as min(*d_n, n), and n is the capacity the launches
// are sized for.  *keys_out / *vals_out receive the buffers holding the result.  A look-back
// wait that runs out sets kErrTimeout in err (the output is then invalid).  With vk (bits > 0)
// the values are then sorted stably by their view, as a more significant key; no sorted keys
// are then written (*keys_out is null).
void launch_sort(const Launch& L, uint32_t* keys, uint32_t* vals, uint32_t* keys_alt, uint32_t* vals_alt,
                 uint32_t n, int key_bits, uint32_t* hist, uint32_t* status, uint32_t* counters, uint32_t* err,
                 uint32_t** keys_out, uint32_t** vals_out, const uint32_t* d_n = nullptr, SortCtl ctl = SortCtl{},
                 const ViewKey* vk = nullptr);

// Sets the sort kernels' launch attributes; call before a stream capture that contains a sort.
void sort_prepare();

// K3b: pair offsets in depth order, poff[i] = sum_{j<i} ntile[order[j]] for i <= n (n =
// min(*d_n, n) if d_n), and *total = min(poff[n], cap).  parts: scratch of
// tile_scan_parts(n) words.
void launch_tile_scan(const Launch& L, const uint32_t* order, const uint32_t* ntile, uint32_t n, const uint32_t* d_n,
                      uint32_t* poff, uint32_t* parts, uint32_t cap, uint32_t* total, uint32_t* err);

// Kernels that read sorted values as indices return at once after a sort timed out (the
// sorted arrays are then not permutations).
// Debug builds: i < n, else the failure is recorded (see kErrBounds) and false returned.
__device__ __forceinline__ bool in_bounds(uint64_t i, uint64_t n, uint32_t* err, DbgSite site) {
    if constexpr (!kDebugChecks) {
        return true;
    } else {
        if (i < n) return true;
        if (err && (atomicOr(err, kErrBounds) & kErrBounds) == 0) {
            err[kDbgWord] = (uint32_t)site;
            *reinterpret_cast<unsigned long long*>(err + kDbgWord + 2) = i;
            *reinterpret_cast<unsigned long long*>(err + kDbgWord + 4) = n;
        }
        return false;
    }
}

__device__ __forceinline__ bool sort_failed(const uint32_t* err) { return (*(volatile const uint32_t*)err & kErrTimeout) != 0; }
size_t tile_scan_parts(uint32_t n);

// K3c: the (tile, instance) pairs of the depth-ordered instances, instance by instance in
// that order and each instance's tiles in row-major order: keys = tile within the group (bits
// 0..23) | sub-tile mask << 24, values = instance index.  Pairs at or beyond cap are not
// written (kErrCapacity).
void launch_pairs(const Launch& L, const ViewDesc* views, int K, const uint32_t* order, const uint32_t* poff,
                  const Record* records, const InstInfo* info, uint32_t n, const uint32_t* d_n, const Params& P,
                  uint32_t* tkeys, uint32_t* tvals, uint32_t cap);

// K4: [start, end) of every tile's run in the tile-sorted keys (d_n: device pair count); the
// tile is the key's low kTileBits bits.
// K4: ranges[tile of the group] = [first, last) entry of its run.  Keys are view in group <<
// P.tbits | tile in its view (bits 0..23); a key whose view is not below nv (dead pairs) has no
// tile.
void launch_ranges(const Launch& L, const uint32_t* keys, uint32_t n, uint2* ranges, int n_tiles,
                   const uint32_t* d_n, const ViewDesc* views, int nv, const Params& P);

// K5: keys/vals are the tile-sorted pairs (each key's sub-tile mask selects the warps that
// stage the instance).
// Checkpoints of the compositor's per-pixel state, for an adjoint that replays the segments of
// long tile lists in parallel (kept lists only).  A tile's list is cut into segments of
// kSegEntries entries; at the start of every segment after the first, the forward warp of each
// sub-tile stores its pixels' state, and at its end how many segments it entered.  The adjoint
// replays each (tile, segment) job from the state the forward had there, so every job takes the
// forward's FP32 decisions exactly as one sequential replay would.
constexpr int kSegChunks = 16;                              // 32-entry chunks per segment
constexpr uint32_t kSegEntries = 32u * (uint32_t)kSegChunks;
struct CkState {
    float T, c0, c1, c2, d, done;                           // transmittance, RGB and depth sums
};
struct Checkpoints {
    CkState* st = nullptr;          // [slot][sub-tile][lane]; null: no checkpoints
    uint32_t* off = nullptr;        // per tile: its first slot (segment s > 0 -> slot off + s - 1)
    uint32_t* last = nullptr;       // per (tile, sub-tile): segments its forward warp entered
    uint2* jobs = nullptr;          // (tile, segment) jobs, longest first
    uint32_t* n_jobs = nullptr;     // device count of jobs
};

void launch_composite(const Launch& L, const ViewDesc* views, int v0, int n_group_views, int n_tiles,
                      const uint2* ranges, const uint32_t* keys, const uint32_t* vals, const Record* records,
                      const Params& P, float* out_rgb, float* out_depth, float* out_alpha, unsigned long long* work,
                      const uint32_t* tile_order = nullptr, const Checkpoints& ck = Checkpoints{});

// The (tile, segment) jobs of a group's lists, longest first, and each tile's first checkpoint
// slot (one block; groups of at most kOrderMaxTiles tiles).
void launch_segment_jobs(const Launch& L, const uint2* ranges, int n_tiles, const Checkpoints& ck);

// The group's tiles in descending order of list length (the compositors' block -> tile map), for
// groups of at most kOrderMaxTiles tiles: with more, the many waves of blocks balance the SMs
// without it.
constexpr int kOrderMaxTiles = 32768;
// Warps per compositor block (forward and adjoint): each warp one 8x4 sub-tile of the block's
// tile; a tile of tile_w x tile_h pixels spans tile_w * tile_h / (32 kCompWarps) blocks.
constexpr int kCompWarps = 2;
void launch_tile_order(const Launch& L, const uint2* ranges, int n_tiles, uint32_t* order);

// Image randomisation of an RGB batch in place (the separate form of the compositor's
// epilogue).  spans[V]: per view its first output pixel, its first quad in the view-by-view
// enumeration of the 4-pixel quads (of the global pixel index) that hold its pixels, and its
// size; n_quads = total quads.
struct AugSpan {
    int64_t pix_off;
    int64_t q0;
    int32_t W, H;
};
void launch_augment(const Launch& L, const AugSpan* spans, int V, int64_t n_quads, const dgs_augment* aug,
                    const uint8_t* overlay, int ow, int oh, float* rgb);

// LiDAR (csrc/lidar.cu).  Per node: records (4 float4 per Gaussian: mean + opacity, whitening
// matrix) and an implicit BVH of 2P boxes (2 float4 each, heap numbering from 1).
struct LidarTreeDev {
    const float4* box;
    const float4* rec;
    int64_t n;
    int64_t P;               // leaves (a power of two; leaf k covers Gaussians 8(k-P) .. +8)
    uint32_t gbase;          // global id of the node's first Gaussian
};
struct LidarSensorDev {
    int32_t env;
    float pose[12];          // world_from_sensor
};
struct LidarSlot {           // per (sensor, slot): sensor in the node's frame
    float R[9];              // node_from_sensor rotation
    float o[3];              // sensor origin in the node frame
    int32_t node;            // -1 = empty slot or invalid pose
    int32_t pad;
};
struct LidarParams {
    float r_min, r_max, alpha_min, alpha_max, t_min, q_max;
};
size_t lidar_tree_nodes(int64_t n);
void launch_lidar_records(const Launch& L, const NodeDesc& nd, float q_max, float4* rec, float4* box, int64_t P);
size_t lidar_level_job_bytes();
void lidar_level_job(void* jobs, int i, float4* box, int64_t first);
void launch_lidar_level(const Launch& L, const void* jobs, int n_jobs, int64_t h, int64_t total);
void launch_lidar_setup(const Launch& L, const LidarSensorDev* sensors, int S, const int32_t* slot_node, int K,
                        const float* node_poses, LidarSlot* out, uint32_t* err);
void launch_lidar_trace(const Launch& L, const LidarTreeDev* trees, const LidarSlot* slots, int K, const float* dirs,
                        int n_dirs, int64_t n_rays, const LidarParams& LP, float* out_d, float* out_a, uint32_t* err,
                        unsigned long long* next_ray);

// Mesh -> Gaussian transfer (csrc/mesh.cu): one Gaussian per facet into node-layout arrays
// (quat must be 16-byte aligned).
void launch_mesh_gaussians(const Launch& L, const float* v, int64_t n_v, const int32_t* f, int64_t n_f,
                           const float* col, float flatten, float opacity_logit, int n_coef, float* mean,
                           float* log_scale, float* quat, float* opac, float* sh, uint32_t* err);

// Depth -> TSDF fusion (csrc/tsdf.cu).
struct TsdfView {
    float R[9], t[3];        // cam_from_world
    float fx, fy, cx, cy;
    int32_t W, H;
    int64_t pix_off;         // first pixel of the view in the depth / coverage arrays
    int64_t q0;              // first pixel of the view in the packed normalised-depth scratch
};
struct TsdfParams {
    float ox, oy, oz, voxel, trunc, inv_trunc, max_weight, min_alpha;
};
void launch_tsdf(const Launch& L, float* F, float* W, int nx, int ny, int64_t n_vox, const TsdfParams& TP,
                 const TsdfView* views, int V, const float* depth, const float* alpha, float* dn, int64_t n_pix);

void launch_composite_bwd(const Launch& L, const ViewDesc* views, int v0, int n_group_views, int n_tiles,
                          const uint2* ranges, const uint32_t* keys, const uint32_t* vals, const Record* records,
                          const Params& P,
                          const float* out_rgb, const float* out_depth, const float* g_rgb, const float* g_depth,
                          float* inst_grad, unsigned long long* n_red = nullptr, const uint32_t* tile_order = nullptr,
                          const Checkpoints& ck = Checkpoints{}, uint32_t n_jobs_bound = 0);

void launch_project_bwd(const Launch& L, int dtype_mask, const NodeDesc* nodes, int n_nodes, const ViewDesc* views,
                        const VNode* vnodes, int K, const float* node_poses, const InstInfo* info,
                        const float* inst_grad, uint32_t n_inst, const Params& P, const dgs_node_grads* grads,
                        float* grad_poses);

// se(3) twists (rho, phi) [n,6] of n poses [n,12] and their 3x4 gradients [n,12].
void launch_pose_twist(const Launch& L, const float* poses, const float* grads, int64_t n, float* out);

size_t sort_status_words(uint32_t n);
int sort_passes(int key_bits);
// Streaming multiprocessors of the current device (read once per process and device).
uint32_t sm_count();

}  // namespace dgs
