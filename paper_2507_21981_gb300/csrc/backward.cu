// Adjoint of the renderer: compositing (K7) and projection + colour + node pose (K8).
//
// Sec. IV: the 3DGS assets are optimised against rendered images and depth, which needs the
// gradient of the renderer with respect to every Gaussian attribute; the rigid node poses of
// Sec. III-B are differentiated the same way.  L = sum g_C . RGB + sum g_D . D.
//
// K7 replays every pixel front to back with exactly the forward's FP32 decisions, keeping only
// the forward outputs: with prefix P_i = sum_{j<=i} w_j c_j, the colour behind Gaussian i
// (normalised, background included) is S_i = (C_out - P_i) / T_{i+1}, and
//   dL/dalpha_i = T_i [ g_C . (c_i - S_i) + g_D (z_i - SD_i) ],
//   dL/dc_i = w_i g_C,  dL/dz_i = w_i g_D,
// because T_{i+1} / (1 - alpha_i) = T_i.  alpha = min(alpha_max, o e^{-q/2}) then gives the
// partials of o and of q = qa (dx + qb dy)^2 + qc dy^2 (zero where alpha is clamped).  Each warp
// reduces its 32 pixels' partials of a record and adds them to the record's 10 accumulators.
//
// K8 recomputes one instance's projection and applies the chain rule through the factored
// quadratic form, the 2D covariance A diag(s^2) A^T + lowpass I (A = J M_R R), the guarded
// Jacobian, the camera_from_node transform, the quaternion normalisation, the sigmoid and the
// real SH basis; the node pose receives the partials of M = Wc [Rn | tn] and of the camera
// centre expressed in the node frame (the SH direction).
#include "dgs_internal.cuh"

namespace dgs {
namespace {

// per-instance partials, in this order
enum { G_U = 0, G_V, G_QA, G_QB, G_QC, G_OP, G_R, G_G, G_B, G_Z, G_N };

// Warp sums of 16 values by recursive halving: at the step with offset o each lane keeps the
// half of its values that its side of the butterfly owns and adds the partner's copy of them
// (8 + 4 + 2 + 1 + 1 shuffles instead of 16 x 5).  Lanes 2j and 2j + 1 end with the total of
// value j.
__device__ __forceinline__ float warp_transpose_sum16(const float (&v)[16], int lane) {
    const uint32_t full = 0xffffffffu;
    float a[8], b[4], c[2];
    const bool h16 = (lane >> 4) & 1, h8 = (lane >> 3) & 1, h4 = (lane >> 2) & 1, h2 = (lane >> 1) & 1;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const float mine = h16 ? v[8 + j] : v[j], give = h16 ? v[j] : v[8 + j];
        a[j] = mine + __shfl_xor_sync(full, give, 16);
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const float mine = h8 ? a[4 + j] : a[j], give = h8 ? a[j] : a[4 + j];
        b[j] = mine + __shfl_xor_sync(full, give, 8);
    }
#pragma unroll
    for (int j = 0; j < 2; ++j) {
        const float mine = h4 ? b[2 + j] : b[j], give = h4 ? b[j] : b[2 + j];
        c[j] = mine + __shfl_xor_sync(full, give, 4);
    }
    const float mine = h2 ? c[1] : c[0], give = h2 ? c[0] : c[1];
    const float d = mine + __shfl_xor_sync(full, give, 2);
    return d + __shfl_xor_sync(full, d, 1);
}

// ------------------------------------------------------------------ K7
__global__ void __launch_bounds__(kCompWarps * 32) k_composite_bwd(const ViewDesc* __restrict__ views, int v0, int nv,
                                                       const uint2* __restrict__ ranges, const uint32_t* __restrict__ keys,
                                                       const uint32_t* __restrict__ vals,
                                                       const Record* __restrict__ rec, Params P,
                                                       const float* __restrict__ out_rgb,
                                                       const float* __restrict__ out_depth,
                                                       const float* __restrict__ g_rgb,
                                                       const float* __restrict__ g_depth, float* __restrict__ ig,
                                                       unsigned long long* __restrict__ n_red,
                                                       const uint32_t* __restrict__ tile_order, Checkpoints ck) {
    __shared__ float4 s_rec[kCompWarps][3][32];
    __shared__ uint32_t s_idx[kCompWarps][32];
    if (sort_failed(P.err)) return;
    const int bpt = (P.tile_w * P.tile_h) / (32 * kCompWarps);   // blocks per tile, as the forward
    const int tb = (int)blockIdx.x / bpt;
    // with checkpoints a block replays one segment of one tile's list (jobs longest first),
    // else the whole list of a tile
    int gt;
    uint32_t seg = 0;
    if (ck.st) {
        if ((uint32_t)tb >= *ck.n_jobs) return;
        const uint2 job = ck.jobs[tb];
        gt = (int)job.x;
        seg = job.y;
    } else {
        gt = tile_order ? (int)tile_order[tb] : tb;
    }
    const int ga = gt + P.tile0;
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
    const int sub_cols = P.tile_w >> 3;
    const int wx0 = tx * P.tile_w + (w % sub_cols) * 8, wy0 = ty * P.tile_h + (w / sub_cols) * 4;
    const int wx1 = min(wx0 + 7, vd.W - 1), wy1 = min(wy0 + 3, vd.H - 1);
    if (wx0 > wx1 || wy0 > wy1) return;
    const int px = wx0 + (lane & 7), py = wy0 + (lane >> 3);
    const bool inside = px < vd.W && py < vd.H;
    const float fx = (float)px + 0.5f, fy = (float)py + 0.5f;
    float gC0 = 0.f, gC1 = 0.f, gC2 = 0.f, gD = 0.f, Co0 = 0.f, Co1 = 0.f, Co2 = 0.f, Do = 0.f;
    if (inside) {
        const int64_t p = vd.pix_off + (int64_t)py * vd.W + px;
        gC0 = g_rgb[p * 3 + 0]; gC1 = g_rgb[p * 3 + 1]; gC2 = g_rgb[p * 3 + 2];
        gD = g_depth ? g_depth[p] : 0.f;
        Co0 = out_rgb[p * 3 + 0]; Co1 = out_rgb[p * 3 + 1]; Co2 = out_rgb[p * 3 + 2];
        Do = out_depth[p];
    }
    if (__all_sync(0xffffffffu, gC0 == 0.f && gC1 == 0.f && gC2 == 0.f && gD == 0.f)) return;
    uint2 range = ranges[gt];
    uint32_t reds = 0;
    float T = 1.f, P0 = 0.f, P1 = 0.f, P2 = 0.f, PD = 0.f;
    bool done = !inside;
    if (ck.st) {
        const int n_sub = P.tile_w * P.tile_h / 32;
        range.x += seg * kSegEntries;
        range.y = min(range.y, range.x + kSegEntries);
        if (seg > 0) {
            // the forward warp's state where this segment starts, or nothing to do if it ended before
            if (seg >= ck.last[(size_t)gt * n_sub + w]) return;
            const CkState c = ck.st[((size_t)(ck.off[gt] + seg - 1) * n_sub + w) * 32 + lane];
            T = c.T; P0 = c.c0; P1 = c.c1; P2 = c.c2; PD = c.d;
            done = c.done != 0.f;
        }
    }
    const uint32_t lt = (1u << lane) - 1u;
    const uint32_t wbit = 1u << (kTileBits + w);
    float4* const sr0 = s_rec[bw][0];
    float4* const sr1 = s_rec[bw][1];
    float4* const sr2 = s_rec[bw][2];
    for (uint32_t base = range.x; base < range.y; base += 32) {
        if (__all_sync(0xffffffffu, done)) break;
        const uint32_t i = base + lane;
        // the forward pass's staging: entries whose sub-tile mask holds this warp's bit
        const bool sel = i < range.y && (__ldg(keys + i) & wbit);
        // (debug builds check every entry of the range, whichever sub-tiles it reaches)
        const bool chk = kDebugChecks && i < range.y;
        const uint32_t idx = sel || chk ? __ldg(vals + i) : 0u;
        const bool rel = sel && (!chk || in_bounds(idx, P.n_rec, P.err, kSiteBackwardRecord));
        const uint32_t m = __ballot_sync(0xffffffffu, rel);
        if (m == 0) continue;
        if (rel) {
            // staged as the forward stages them: the threshold and the scaled qa beside the raw
            // coefficients that the gradients use
            const Record* r = rec + idx;
            const int pos = __popc(m & lt);
            const float4 a = r->r0, q = r->r1, col = r->r2;
            sr0[pos] = a;
            sr1[pos] = make_float4(q.x, q.y, q.z, reach_threshold(P, a.z));
            sr2[pos] = make_float4(col.x, col.y, col.z, kHalfLog2e * q.x);
            s_idx[bw][pos] = idx;
        }
        __syncwarp();
        const int n = __popc(m);
        for (int k = 0; k < n; ++k) {
            // the forward pass's decisions, without branches: same staged products, same exponent
            const float4 g0 = sr0[k], g1 = sr1[k], g2 = sr2[k];
            const float dx = fx - g0.x, dy = fy - g0.y;
            float t;
            const float pe = pixel_exponent(g2.w, g1.y, kHalfLog2e * g1.z, dx, dy, t);
            const bool hit = !done && pe >= g1.w;
            const float ex = fast_exp2(pe);
            const float a_raw = g0.z * ex;
            const float alpha = fminf(P.alpha_max, a_raw);
            const float Tn = fmaf(-alpha, T, T);       // T (1 - alpha), one rounding
            const bool stop = hit && Tn < P.t_min;
            const bool contrib = hit && !stop;
            done = done || stop;
            float g[G_N];
#pragma unroll
            for (int e = 0; e < G_N; ++e) g[e] = 0.f;
            if (contrib) {
                const float wgt = alpha * T;
                P0 = fmaf(wgt, g2.x, P0); P1 = fmaf(wgt, g2.y, P1); P2 = fmaf(wgt, g2.z, P2);
                PD = fmaf(wgt, g0.w, PD);
                const float iTn = __fdividef(1.f, Tn);   // Tn >= t_min > 0
                const float S0 = (Co0 - P0) * iTn, S1 = (Co1 - P1) * iTn, S2 = (Co2 - P2) * iTn;
                const float SD = (Do - PD) * iTn;
                const float dal = T * (gC0 * (g2.x - S0) + gC1 * (g2.y - S1) + gC2 * (g2.z - S2) + gD * (g0.w - SD));
                g[G_R] = wgt * gC0; g[G_G] = wgt * gC1; g[G_B] = wgt * gC2; g[G_Z] = wgt * gD;
                if (!(a_raw > P.alpha_max)) {
                    g[G_OP] = dal * ex;
                    const float dq = -0.5f * alpha * dal;
                    g[G_QA] = dq * t * t;
                    g[G_QB] = dq * 2.f * g1.x * t * dy;
                    g[G_QC] = dq * dy * dy;
                    g[G_U] = dq * (-2.f * g1.x * t);
                    g[G_V] = dq * (-2.f * fmaf(g1.x * t, g1.y, g1.z * dy));
                }
                T = Tn;
            }
            if (__ballot_sync(0xffffffffu, contrib) == 0) continue;
            const uint32_t r = s_idx[bw][k];
            float v16[16];
#pragma unroll
            for (int e = 0; e < 16; ++e) v16[e] = e < G_N ? g[e] : 0.f;
            const float tot = warp_transpose_sum16(v16, lane);
            const int e = lane >> 1;
            const bool add = (lane & 1) == 0 && e < G_N && tot != 0.f;
            if (add) atomicAdd(ig + (size_t)r * G_N + e, tot);
            if (n_red) reds += __popc(__ballot_sync(0xffffffffu, add));
        }
        __syncwarp();
    }
    if (n_red && lane == 0 && reds) atomicAdd(n_red, (unsigned long long)reds);
}

// ------------------------------------------------------------------ K8
__device__ __forceinline__ void sh_basis_grad(int deg, float x, float y, float z, float Y[16], float dY[16][3]) {
    constexpr float kY00 = 0.28209479177387814f, kC1 = 0.4886025119029199f;
    constexpr float kC2a = 1.0925484305920792f, kC2b = 0.31539156525252005f, kC2c = 0.5462742152960396f;
    constexpr float kC3a = 0.5900435899266435f, kC3b = 2.890611442640554f, kC3c = 0.4570457994644658f;
    constexpr float kC3d = 0.3731763325901154f, kC3e = 1.445305721320277f;
#pragma unroll
    for (int k = 0; k < 16; ++k) { Y[k] = 0.f; dY[k][0] = dY[k][1] = dY[k][2] = 0.f; }
    Y[0] = kY00;
    if (deg < 1) return;
    Y[1] = -kC1 * y; dY[1][1] = -kC1;
    Y[2] = kC1 * z;  dY[2][2] = kC1;
    Y[3] = -kC1 * x; dY[3][0] = -kC1;
    if (deg < 2) return;
    const float xx = x * x, yy = y * y, zz = z * z;
    Y[4] = kC2a * x * y;        dY[4][0] = kC2a * y; dY[4][1] = kC2a * x;
    Y[5] = -kC2a * y * z;       dY[5][1] = -kC2a * z; dY[5][2] = -kC2a * y;
    Y[6] = kC2b * (3.f * zz - 1.f); dY[6][2] = 6.f * kC2b * z;
    Y[7] = -kC2a * x * z;       dY[7][0] = -kC2a * z; dY[7][2] = -kC2a * x;
    Y[8] = kC2c * (xx - yy);    dY[8][0] = 2.f * kC2c * x; dY[8][1] = -2.f * kC2c * y;
    if (deg < 3) return;
    Y[9] = -kC3a * y * (3.f * xx - yy);  dY[9][0] = -6.f * kC3a * x * y; dY[9][1] = -3.f * kC3a * (xx - yy);
    Y[10] = kC3b * x * y * z;            dY[10][0] = kC3b * y * z; dY[10][1] = kC3b * x * z; dY[10][2] = kC3b * x * y;
    Y[11] = -kC3c * y * (5.f * zz - 1.f); dY[11][1] = -kC3c * (5.f * zz - 1.f); dY[11][2] = -10.f * kC3c * y * z;
    Y[12] = kC3d * z * (5.f * zz - 3.f);  dY[12][2] = kC3d * (15.f * zz - 3.f);
    Y[13] = -kC3c * x * (5.f * zz - 1.f); dY[13][0] = -kC3c * (5.f * zz - 1.f); dY[13][2] = -10.f * kC3c * x * z;
    Y[14] = kC3e * z * (xx - yy);        dY[14][0] = 2.f * kC3e * x * z; dY[14][1] = -2.f * kC3e * y * z; dY[14][2] = kC3e * (xx - yy);
    Y[15] = -kC3a * x * (xx - 3.f * yy); dY[15][0] = -3.f * kC3a * (xx - yy); dY[15][1] = 6.f * kC3a * x * y;
}

__device__ __forceinline__ int node_of_gid(const NodeDesc* nodes, int n_nodes, uint32_t gid) {
    int lo = 0, hi = n_nodes - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if ((uint64_t)nodes[mid].gbase <= gid) lo = mid; else hi = mid - 1;
    }
    // nodes with no Gaussians share gbase with the next node: step back to a non-empty one
    while (lo > 0 && nodes[lo].n == 0) --lo;
    return lo;
}

// Colour adjoint of one instance at SH degree DEG, known at compile time so that the basis and
// its gradient stay in registers: rgb = max(0, sum_c Y_c(d) sh_c + 1/2) per channel; adds the
// SH coefficients' gradients (where the channel is not clamped) and the direction gradient gd.
template <int DEG, int DT>
__device__ __forceinline__ void sh_colour_bwd(const NodeDesc& nd, int64_t i, float dx, float dy, float dz,
                                              const float (&gcol)[3], float* gsh, float (&gd)[3]) {
    constexpr int NC = (DEG + 1) * (DEG + 1);
    float Y[16], dY[16][3];
    sh_basis_grad(DEG, dx, dy, dz, Y, dY);
    const int64_t sb = i * NC * 3;
    float raw[3] = {0.5f, 0.5f, 0.5f};
#pragma unroll
    for (int c = 0; c < NC; ++c)
#pragma unroll
        for (int ch = 0; ch < 3; ++ch) raw[ch] = fmaf(Y[c], ld_attr<DT>(nd.sh, sb + c * 3 + ch), raw[ch]);
#pragma unroll
    for (int c = 0; c < NC; ++c) {
#pragma unroll
        for (int ch = 0; ch < 3; ++ch) {
            if (!(raw[ch] > 0.f) || gcol[ch] == 0.f) continue;
            if (gsh) atomicAdd(gsh + sb + c * 3 + ch, gcol[ch] * Y[c]);
            const float cf = gcol[ch] * ld_attr<DT>(nd.sh, sb + c * 3 + ch);
            gd[0] = fmaf(cf, dY[c][0], gd[0]); gd[1] = fmaf(cf, dY[c][1], gd[1]); gd[2] = fmaf(cf, dY[c][2], gd[2]);
        }
    }
}

template <int DT>
__global__ void __launch_bounds__(128, 5) k_project_bwd(const NodeDesc* __restrict__ nodes, int n_nodes,
                                                     const ViewDesc* __restrict__ views,
                                                     const VNode* __restrict__ vnodes, int K,
                                                     const float* __restrict__ node_poses,
                                                     const InstInfo* __restrict__ info, const float* __restrict__ ig,
                                                     uint32_t n_inst, Params P, const dgs_node_grads* __restrict__ grads,
                                                     float* __restrict__ grad_poses) {
    const uint32_t r = blockIdx.x * blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31;
    bool act = r < n_inst;
    int k = 0, vv = -1;
    int64_t i = 0;
    if (act) {
        const InstInfo inf = info[r];
        vv = (int)inf.view;
        k = node_of_gid(nodes, n_nodes, inf.gid);
        i = (int64_t)inf.gid - nodes[k].gbase;
        act = nodes[k].dtype == DT && in_bounds((uint64_t)i, (uint64_t)nodes[k].n, P.err, kSiteProjectBwdGaussian);
    }
    if (act) {
        // an instance that no pixel composited adds nothing -- and a dead record of the count
        // pass's conservative cull (never composited) may have a degenerate projection whose
        // recomputed Jacobian would turn its zero partials into NaN
        const float* pg = ig + (size_t)r * G_N;
        bool any = false;
#pragma unroll
        for (int e = 0; e < G_N; ++e) any |= pg[e] != 0.f;
        act = any;
    }
    float gRn[9], gtn[3];
#pragma unroll
    for (int e = 0; e < 9; ++e) gRn[e] = 0.f;
    gtn[0] = gtn[1] = gtn[2] = 0.f;
    if (act) {
        const NodeDesc& nd = nodes[k];
        const VNode& vn = vnodes[vv];
        const ViewDesc& vd = views[vv / K];
        const float* M = vn.M;
        const float* pg = ig + (size_t)r * G_N;
        const float gu = pg[G_U], gv = pg[G_V], gqa = pg[G_QA], gqb = pg[G_QB], gqc = pg[G_QC];
        const float gop = pg[G_OP], gcr = pg[G_R], gcg = pg[G_G], gcb = pg[G_B], gz = pg[G_Z];
        // ---------------------------------------------------------------- recompute the forward
        const float mx = __ldg(nd.mean + i * 3 + 0), my = __ldg(nd.mean + i * 3 + 1), mz = __ldg(nd.mean + i * 3 + 2);
        const float s0 = __expf(2.f * ld_attr<DT>(nd.log_scale, i * 3 + 0));
        const float s1 = __expf(2.f * ld_attr<DT>(nd.log_scale, i * 3 + 1));
        const float s2 = __expf(2.f * ld_attr<DT>(nd.log_scale, i * 3 + 2));
        const float q0 = ld_attr<DT>(nd.quat, i * 4 + 0), q1 = ld_attr<DT>(nd.quat, i * 4 + 1);
        const float q2 = ld_attr<DT>(nd.quat, i * 4 + 2), q3 = ld_attr<DT>(nd.quat, i * 4 + 3);
        const float qinv = rsqrtf(q0 * q0 + q1 * q1 + q2 * q2 + q3 * q3);
        const float w_ = q0 * qinv, x_ = q1 * qinv, y_ = q2 * qinv, z_ = q3 * qinv;
        float R[3][3];
        R[0][0] = 1.f - 2.f * (y_ * y_ + z_ * z_); R[0][1] = 2.f * (x_ * y_ - w_ * z_); R[0][2] = 2.f * (x_ * z_ + w_ * y_);
        R[1][0] = 2.f * (x_ * y_ + w_ * z_); R[1][1] = 1.f - 2.f * (x_ * x_ + z_ * z_); R[1][2] = 2.f * (y_ * z_ - w_ * x_);
        R[2][0] = 2.f * (x_ * z_ - w_ * y_); R[2][1] = 2.f * (y_ * z_ + w_ * x_); R[2][2] = 1.f - 2.f * (x_ * x_ + y_ * y_);
        const float s[3] = {s0, s1, s2};
        const float z = camera_depth(vn, mx, my, mz);
        const float tx = camera_row(vn, 0, mx, my, mz);
        const float ty = camera_row(vn, 1, mx, my, mz);
        const float iz = 1.f / z;
        const float xr = tx * iz, yr = ty * iz;
        const bool clx = xr > vd.limx || xr < -vd.limx, cly = yr > vd.limy || yr < -vd.limy;
        const float xc = fminf(vd.limx, fmaxf(-vd.limx, xr)), yc = fminf(vd.limy, fmaxf(-vd.limy, yr));
        const float fxz = vd.fx * iz, fyz = vd.fy * iz;
        float Tm[2][3];
        Tm[0][0] = fxz * fmaf(-xc, M[8], M[0]); Tm[0][1] = fxz * fmaf(-xc, M[9], M[1]); Tm[0][2] = fxz * fmaf(-xc, M[10], M[2]);
        Tm[1][0] = fyz * fmaf(-yc, M[8], M[4]); Tm[1][1] = fyz * fmaf(-yc, M[9], M[5]); Tm[1][2] = fyz * fmaf(-yc, M[10], M[6]);
        float A[2][3];
#pragma unroll
        for (int a = 0; a < 2; ++a)
#pragma unroll
            for (int c = 0; c < 3; ++c) A[a][c] = Tm[a][0] * R[0][c] + Tm[a][1] * R[1][c] + Tm[a][2] * R[2][c];
        const float cxx = s0 * A[0][0] * A[0][0] + s1 * A[0][1] * A[0][1] + s2 * A[0][2] * A[0][2] + P.lowpass;
        const float cxy = s0 * A[0][0] * A[1][0] + s1 * A[0][1] * A[1][1] + s2 * A[0][2] * A[1][2];
        const float cyy = s0 * A[1][0] * A[1][0] + s1 * A[1][1] * A[1][1] + s2 * A[1][2] * A[1][2] + P.lowpass;
        const float m01 = A[0][0] * A[1][1] - A[0][1] * A[1][0], m02 = A[0][0] * A[1][2] - A[0][2] * A[1][0];
        const float m12 = A[0][1] * A[1][2] - A[0][2] * A[1][1];
        const float det = s0 * s1 * m01 * m01 + s0 * s2 * m02 * m02 + s1 * s2 * m12 * m12 +
                          P.lowpass * (cxx + cyy - P.lowpass);
        const float idet = 1.f / det, icyy = 1.f / cyy;
        const float op = 1.f / (1.f + __expf(-__ldg(nd.opac + i)));
        // ---------------------------------------------------------------- opacity
        const float glogit = gop * op * (1.f - op);
        // ---------------------------------------------------------------- colour (SH in the node frame)
        float gmu[3] = {0.f, 0.f, 0.f};
        float go[3] = {0.f, 0.f, 0.f};
        {
            float dx = mx - vn.o[0], dy = my - vn.o[1], dz = mz - vn.o[2];
            const float dlen_inv = rsqrtf(dx * dx + dy * dy + dz * dz);
            dx *= dlen_inv; dy *= dlen_inv; dz *= dlen_inv;
            const float gcol[3] = {gcr, gcg, gcb};
            float gd[3] = {0.f, 0.f, 0.f};
            float* gsh = grads[k].sh;
            switch (nd.deg) {
                case 0: sh_colour_bwd<0, DT>(nd, i, dx, dy, dz, gcol, gsh, gd); break;
                case 1: sh_colour_bwd<1, DT>(nd, i, dx, dy, dz, gcol, gsh, gd); break;
                case 2: sh_colour_bwd<2, DT>(nd, i, dx, dy, dz, gcol, gsh, gd); break;
                default: sh_colour_bwd<3, DT>(nd, i, dx, dy, dz, gcol, gsh, gd); break;
            }
            const float dd = gd[0] * dx + gd[1] * dy + gd[2] * dz;
            const float gdir[3] = {(gd[0] - dx * dd) * dlen_inv, (gd[1] - dy * dd) * dlen_inv, (gd[2] - dz * dd) * dlen_inv};
#pragma unroll
            for (int a = 0; a < 3; ++a) { gmu[a] += gdir[a]; go[a] = -gdir[a]; }
        }
        // ---------------------------------------------------------------- factored form -> 2D covariance
        const float idet2 = idet * idet;
        const float gcxx = gqa * (-cyy * cyy * idet2);
        const float gcxy = gqa * (2.f * cxy * cyy * idet2) - gqb * icyy;
        const float gcyy = gqa * (-cxy * cxy * idet2) + gqb * cxy * icyy * icyy - gqc * icyy * icyy;
        // Sigma2D = A S A^T + lp I, G = [[gcxx, gcxy/2], [gcxy/2, gcyy]]
        float gA[2][3];
        float gls[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const float a0 = A[0][c], a1 = A[1][c];
            gA[0][c] = 2.f * s[c] * (gcxx * a0 + 0.5f * gcxy * a1);
            gA[1][c] = 2.f * s[c] * (0.5f * gcxy * a0 + gcyy * a1);
            gls[c] = 2.f * s[c] * (gcxx * a0 * a0 + gcxy * a0 * a1 + gcyy * a1 * a1);
        }
        // A = T R
        float gT[2][3], gR[3][3];
#pragma unroll
        for (int a = 0; a < 2; ++a)
#pragma unroll
            for (int j = 0; j < 3; ++j) gT[a][j] = gA[a][0] * R[j][0] + gA[a][1] * R[j][1] + gA[a][2] * R[j][2];
#pragma unroll
        for (int j = 0; j < 3; ++j)
#pragma unroll
            for (int c = 0; c < 3; ++c) gR[j][c] = Tm[0][j] * gA[0][c] + Tm[1][j] * gA[1][c];
        // R(q) -> normalised q -> q
        float gqn[4];
        gqn[0] = 2.f * (-z_ * gR[0][1] + y_ * gR[0][2] + z_ * gR[1][0] - x_ * gR[1][2] - y_ * gR[2][0] + x_ * gR[2][1]);
        gqn[1] = 2.f * (y_ * gR[0][1] + z_ * gR[0][2] + y_ * gR[1][0] - 2.f * x_ * gR[1][1] - w_ * gR[1][2] + z_ * gR[2][0] +
                        w_ * gR[2][1] - 2.f * x_ * gR[2][2]);
        gqn[2] = 2.f * (-2.f * y_ * gR[0][0] + x_ * gR[0][1] + w_ * gR[0][2] + x_ * gR[1][0] + z_ * gR[1][2] - w_ * gR[2][0] +
                        z_ * gR[2][1] - 2.f * y_ * gR[2][2]);
        gqn[3] = 2.f * (-2.f * z_ * gR[0][0] - w_ * gR[0][1] + x_ * gR[0][2] + w_ * gR[1][0] - 2.f * z_ * gR[1][1] +
                        y_ * gR[1][2] + x_ * gR[2][0] + y_ * gR[2][1]);
        const float qd = gqn[0] * w_ + gqn[1] * x_ + gqn[2] * y_ + gqn[3] * z_;
        const float gq[4] = {(gqn[0] - w_ * qd) * qinv, (gqn[1] - x_ * qd) * qinv, (gqn[2] - y_ * qd) * qinv,
                             (gqn[3] - z_ * qd) * qinv};
        // T = J M_R with J = [[fx/z, 0, -fx xc/z], [0, fy/z, -fy yc/z]]
        const float J[2][3] = {{fxz, 0.f, -fxz * xc}, {0.f, fyz, -fyz * yc}};
        float gMR[3][3];
#pragma unroll
        for (int b = 0; b < 3; ++b)
#pragma unroll
            for (int c = 0; c < 3; ++c) gMR[b][c] = J[0][b] * gT[0][c] + J[1][b] * gT[1][c];
        float gJ[2][3];
#pragma unroll
        for (int a = 0; a < 2; ++a)
#pragma unroll
            for (int b = 0; b < 3; ++b) gJ[a][b] = gT[a][0] * M[b * 4 + 0] + gT[a][1] * M[b * 4 + 1] + gT[a][2] * M[b * 4 + 2];
        float gt[3] = {0.f, 0.f, 0.f};
        const float iz2 = iz * iz;
        gt[2] += gJ[0][0] * (-vd.fx * iz2) + gJ[1][1] * (-vd.fy * iz2);
        if (!clx) { gt[2] += gJ[0][2] * (2.f * vd.fx * tx * iz2 * iz); gt[0] += gJ[0][2] * (-vd.fx * iz2); }
        else { gt[2] += gJ[0][2] * (vd.fx * xc * iz2); }
        if (!cly) { gt[2] += gJ[1][2] * (2.f * vd.fy * ty * iz2 * iz); gt[1] += gJ[1][2] * (-vd.fy * iz2); }
        else { gt[2] += gJ[1][2] * (vd.fy * yc * iz2); }
        // u = fx tx/z + cx, v = fy ty/z + cy, depth = z
        gt[0] += gu * vd.fx * iz; gt[2] += -gu * vd.fx * tx * iz2;
        gt[1] += gv * vd.fy * iz; gt[2] += -gv * vd.fy * ty * iz2;
        gt[2] += gz;
        // t = M_R mu + M_t
        const float mu[3] = {mx, my, mz};
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            gmu[a] += M[0 * 4 + a] * gt[0] + M[1 * 4 + a] * gt[1] + M[2 * 4 + a] * gt[2];
#pragma unroll
            for (int b = 0; b < 3; ++b) gMR[a][b] += gt[a] * mu[b];
        }
        // ---------------------------------------------------------------- node pose: M = Wc [Rn | tn] + [0 | tc]
        const float* Wc = vd.cam;
        const float* Pn = node_poses + ((int64_t)vd.env * K + (vv % K)) * 12;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
#pragma unroll
            for (int b = 0; b < 3; ++b) gRn[a * 3 + b] = Wc[0 * 4 + a] * gMR[0][b] + Wc[1 * 4 + a] * gMR[1][b] + Wc[2 * 4 + a] * gMR[2][b];
            gtn[a] = Wc[0 * 4 + a] * gt[0] + Wc[1 * 4 + a] * gt[1] + Wc[2 * 4 + a] * gt[2];
        }
        // camera centre in the node frame: o = Rn^T (o_cam - tn), o_cam = -Wc^T tc
        float oc[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) oc[a] = -(Wc[0 * 4 + a] * Wc[3] + Wc[1 * 4 + a] * Wc[7] + Wc[2 * 4 + a] * Wc[11]);
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const float rel = oc[a] - Pn[a * 4 + 3];
#pragma unroll
            for (int b = 0; b < 3; ++b) gRn[a * 3 + b] += rel * go[b];
            gtn[a] -= Pn[a * 4 + 0] * go[0] + Pn[a * 4 + 1] * go[1] + Pn[a * 4 + 2] * go[2];
        }
        // ---------------------------------------------------------------- Gaussian parameters
        const dgs_node_grads& G = grads[k];
        if (G.mean) { atomicAdd(G.mean + i * 3 + 0, gmu[0]); atomicAdd(G.mean + i * 3 + 1, gmu[1]); atomicAdd(G.mean + i * 3 + 2, gmu[2]); }
        if (G.log_scale) {
            atomicAdd(G.log_scale + i * 3 + 0, gls[0]); atomicAdd(G.log_scale + i * 3 + 1, gls[1]);
            atomicAdd(G.log_scale + i * 3 + 2, gls[2]);
        }
        if (G.quat) {
            atomicAdd(G.quat + i * 4 + 0, gq[0]); atomicAdd(G.quat + i * 4 + 1, gq[1]);
            atomicAdd(G.quat + i * 4 + 2, gq[2]); atomicAdd(G.quat + i * 4 + 3, gq[3]);
        }
        if (G.opacity_logit) atomicAdd(G.opacity_logit + i, glogit);
    }
    // ---------------------------------------------------------------- pose gradient, reduced per warp
    if (!grad_poses) return;
    // the (view, slot) of the first active lane; a warp whose active lanes all share it reduces
    // its pose partials with one transpose-sum instead of 12 atomics per lane
    const uint32_t am = __ballot_sync(0xffffffffu, act);
    const int lead = am ? __shfl_sync(0xffffffffu, vv, __ffs(am) - 1) : -1;
    const bool same = __all_sync(0xffffffffu, !act || vv == lead);
    if (same && lead >= 0) {
        const ViewDesc& vd0 = views[lead / K];
        float* gp = grad_poses + ((int64_t)vd0.env * K + (lead % K)) * 12;
        // the 3x4 pose partials in row-major [R | t] order, summed over the warp
        float v16[16];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
#pragma unroll
            for (int b = 0; b < 3; ++b) v16[a * 4 + b] = gRn[a * 3 + b];
            v16[a * 4 + 3] = gtn[a];
        }
#pragma unroll
        for (int e = 12; e < 16; ++e) v16[e] = 0.f;
        const float tot = warp_transpose_sum16(v16, lane);
        if ((lane & 1) == 0 && (lane >> 1) < 12) atomicAdd(gp + (lane >> 1), tot);
    } else if (act) {
        const ViewDesc& vdl = views[vv / K];
        float* gp = grad_poses + ((int64_t)vdl.env * K + (vv % K)) * 12;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
#pragma unroll
            for (int b = 0; b < 3; ++b) atomicAdd(gp + a * 4 + b, gRn[a * 3 + b]);
            atomicAdd(gp + a * 4 + 3, gtn[a]);
        }
    }
}

// Sec. III-B / IV: se(3) gradient of a rigid pose under a left perturbation.  With
// T' = exp(xi^) T, xi = (rho, phi), to first order R' = R + [phi]x R and t' = t + [phi]x t + rho,
// so dL = G_R : ([phi]x R) + G_t . ([phi]x t) + G_t . rho.  Writing A = G_R R^T + G_t t^T, the
// phi part is sum_ij A_ij ([phi]x)_ij = phi . (A_21 - A_12, A_02 - A_20, A_10 - A_01) (0-based),
// and the rho part is G_t.  One thread per pose.
__global__ void k_pose_twist(const float* __restrict__ poses, const float* __restrict__ grads, int64_t n,
                             float* __restrict__ out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float* T = poses + i * 12;
    const float* G = grads + i * 12;
    float A[3][3];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b)
            A[a][b] = fmaf(G[a * 4 + 0], T[b * 4 + 0], fmaf(G[a * 4 + 1], T[b * 4 + 1], fmaf(G[a * 4 + 2], T[b * 4 + 2],
                                                                                        G[a * 4 + 3] * T[b * 4 + 3])));
    float* o = out + i * 6;
    o[0] = G[3]; o[1] = G[7]; o[2] = G[11];
    o[3] = A[2][1] - A[1][2];
    o[4] = A[0][2] - A[2][0];
    o[5] = A[1][0] - A[0][1];
}

}  // namespace

void launch_pose_twist(const Launch& L, const float* poses, const float* grads, int64_t n, float* out) {
    if (n <= 0) return;
    k_pose_twist<<<(unsigned)((n + 127) / 128), 128, 0, L.stream>>>(poses, grads, n, out);
    ++*L.launches;
}

void launch_composite_bwd(const Launch& L, const ViewDesc* views, int v0, int n_group_views, int n_tiles,
                          const uint2* ranges, const uint32_t* keys, const uint32_t* vals, const Record* records,
                          const Params& P, const float* out_rgb, const float* out_depth, const float* g_rgb,
                          const float* g_depth, float* inst_grad, unsigned long long* n_red,
                          const uint32_t* tile_order, const Checkpoints& ck, uint32_t n_jobs_bound) {
    if (n_tiles == 0) return;
    const int bpt = (P.tile_w * P.tile_h) / (32 * kCompWarps);
    const uint32_t units = ck.st ? n_jobs_bound : (uint32_t)n_tiles;   // jobs beyond the live count exit
    k_composite_bwd<<<units * bpt, kCompWarps * 32, 0, L.stream>>>(views, v0, n_group_views, ranges, keys, vals,
                                                                   records, P, out_rgb, out_depth, g_rgb, g_depth,
                                                                   inst_grad, n_red, tile_order, ck);
    ++*L.launches;
}

void launch_project_bwd(const Launch& L, int dtype_mask, const NodeDesc* nodes, int n_nodes, const ViewDesc* views,
                        const VNode* vnodes, int K, const float* node_poses, const InstInfo* info,
                        const float* inst_grad, uint32_t n_inst, const Params& P, const dgs_node_grads* grads,
                        float* grad_poses) {
    if (n_inst == 0) return;
    const unsigned blocks = (n_inst + 127) / 128;
    if (dtype_mask & (1 << DGS_F32)) {
        k_project_bwd<DGS_F32><<<blocks, 128, 0, L.stream>>>(nodes, n_nodes, views, vnodes, K, node_poses, info, inst_grad,
                                                             n_inst, P, grads, grad_poses);
        ++*L.launches;
    }
    if (dtype_mask & (1 << DGS_BF16)) {
        k_project_bwd<DGS_BF16><<<blocks, 128, 0, L.stream>>>(nodes, n_nodes, views, vnodes, K, node_poses, info, inst_grad,
                                                              n_inst, P, grads, grad_poses);
        ++*L.launches;
    }
    if (dtype_mask & (1 << DGS_F16)) {
        k_project_bwd<DGS_F16><<<blocks, 128, 0, L.stream>>>(nodes, n_nodes, views, vnodes, K, node_poses, info, inst_grad,
                                                             n_inst, P, grads, grad_poses);
        ++*L.launches;
    }
}

}  // namespace dgs
