// Projection and tile binning (kernels K1 and K2 of the renderer).
//
// Sec. III-A ("Renderer"): the native 3DGS pipeline splats every Gaussian by EWA projection
// of its 3D covariance, evaluates its spherical-harmonics colour and bins it to the screen
// tiles it overlaps before depth sorting.  Sec. III-B: interactive nodes carry their own
// rigid pose, so every Gaussian is first moved by its node's world_from_node transform; here
// node pose and camera are composed once per (view, slot) into camera_from_node.
//
// Work decomposition: a warp owns a chunk of 32 consecutive Gaussians of one node.  The
// count pass projects the chunk (no colour) and writes, per (view, chunk), the number of
// visible instances and of (instance, tile) pairs.  After an exclusive scan of that table the
// emit pass projects again, evaluates colour and writes the instance records and sort pairs
// at their scanned offsets.  The order is therefore deterministic: within a view, instances
// and pairs follow the global id, which makes a stable radix sort break depth ties by id.
// Batched mode: a warp loads its Gaussians' attributes once and loops over every view that
// contains the node.  Plain mode: one launch per view, attributes read again for every view.
#include <math.h>

#include "dgs_internal.cuh"

namespace dgs {
namespace {

// ------------------------------------------------------------------ setup: camera_from_node
// One thread per (view, slot).  camera_from_node is composed with compensated sums and kept as
// M + Ml, within about 2^-48 of the exact product of the two FP32 transforms, so that camera
// space points (the depth key and the projected centre) can be faithfully rounded.

// Compensated sum of n products a_k b_k as (hi, lo) with hi = fl(hi + lo).
__device__ __forceinline__ void dot_hi_lo(const float* a, const float* b, int n, float& hi, float& lo) {
    float p, s, h, r, q;
    two_prod(a[0], b[0], p, s);
    for (int k = 1; k < n; ++k) {
        two_prod(a[k], b[k], h, r);
        two_sum(p, h, p, q);
        s = __fadd_rn(s, __fadd_rn(q, r));
    }
    hi = __fadd_rn(p, s);
    lo = __fsub_rn(s, __fsub_rn(hi, p));
}
__global__ void k_setup_views(const ViewDesc* __restrict__ views, int n_views, const float* __restrict__ poses,
                              const int32_t* __restrict__ slot_node, int K, VNode* __restrict__ vnodes,
                              const int64_t* __restrict__ vnode_tab, uint32_t* err) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_views * K) return;
    const int v = i / K, j = i % K;
    const ViewDesc& vd = views[v];
    VNode out;
    out.node = slot_node[i];
    out.tab = vnode_tab[i];
    const float* P = poses + ((int64_t)vd.env * K + j) * 12;
    float R[9], t[3];
    bool bad = false;
    if (out.node >= 0) {
        for (int a = 0; a < 3; ++a) {
            for (int b = 0; b < 3; ++b) R[a * 3 + b] = P[a * 4 + b];
            t[a] = P[a * 4 + 3];
        }
        for (int a = 0; a < 12; ++a) bad |= !isfinite(P[a]);
        // rigidity: R^T R = I within 1e-4
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) {
                float s = R[0 * 3 + a] * R[0 * 3 + b] + R[1 * 3 + a] * R[1 * 3 + b] + R[2 * 3 + a] * R[2 * 3 + b];
                bad |= fabsf(s - (a == b ? 1.f : 0.f)) > 1e-4f;
            }
    } else {
        for (int a = 0; a < 9; ++a) R[a] = (a % 4 == 0) ? 1.f : 0.f;
        t[0] = t[1] = t[2] = 0.f;
    }
    if (bad) atomicOr(err, kErrPose);
    const float* W = vd.cam;   // rows of [Wc | tc]
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 4; ++b) {
            const float wa[4] = {W[a * 4 + 0], W[a * 4 + 1], W[a * 4 + 2], W[a * 4 + 3]};
            const float col[4] = {b < 3 ? R[0 * 3 + b] : t[0], b < 3 ? R[1 * 3 + b] : t[1], b < 3 ? R[2 * 3 + b] : t[2], 1.f};
            dot_hi_lo(wa, col, b < 3 ? 3 : 4, out.M[a * 4 + b], out.Ml[a * 4 + b]);
        }
    // camera centre in the node frame: o = -M_R^T M_t
    for (int b = 0; b < 3; ++b)
        out.o[b] = -(out.M[0 * 4 + b] * out.M[3] + out.M[1 * 4 + b] * out.M[7] + out.M[2 * 4 + b] * out.M[11]);
    vnodes[i] = out;
}

// ------------------------------------------------------------------ per-Gaussian geometry
struct Gauss {
    float mx, my, mz;
    float r00, r01, r02, r10, r11, r12, r20, r21, r22;   // rotation of the unit quaternion
    float s0, s1, s2;                                      // squared scales exp(2 log s)
    float smax;                                            // largest squared scale
};

constexpr int kGeoStride = 17;   // 16 floats of Gauss + 1 pad: conflict-free reads by other lanes

__device__ __forceinline__ void put_geo(float* __restrict__ row, const Gauss& g) {
    row[0] = g.mx; row[1] = g.my; row[2] = g.mz;
    row[3] = g.r00; row[4] = g.r01; row[5] = g.r02; row[6] = g.r10; row[7] = g.r11; row[8] = g.r12;
    row[9] = g.r20; row[10] = g.r21; row[11] = g.r22; row[12] = g.s0; row[13] = g.s1; row[14] = g.s2;
    row[15] = g.smax;
}

__device__ __forceinline__ void get_geo(const float* __restrict__ row, Gauss& g) {
    g.mx = row[0]; g.my = row[1]; g.mz = row[2];
    g.r00 = row[3]; g.r01 = row[4]; g.r02 = row[5]; g.r10 = row[6]; g.r11 = row[7]; g.r12 = row[8];
    g.r20 = row[9]; g.r21 = row[10]; g.r22 = row[11]; g.s0 = row[12]; g.s1 = row[13]; g.s2 = row[14];
    g.smax = row[15];
}

template <int DT>
__device__ __forceinline__ void load_geometry(const NodeDesc& nd, int64_t i, Gauss& g) {
    g.mx = __ldg(nd.mean + i * 3 + 0);
    g.my = __ldg(nd.mean + i * 3 + 1);
    g.mz = __ldg(nd.mean + i * 3 + 2);
    g.s0 = __expf(2.f * ld_attr<DT>(nd.log_scale, i * 3 + 0));
    g.s1 = __expf(2.f * ld_attr<DT>(nd.log_scale, i * 3 + 1));
    g.s2 = __expf(2.f * ld_attr<DT>(nd.log_scale, i * 3 + 2));
    float w = ld_attr<DT>(nd.quat, i * 4 + 0), x = ld_attr<DT>(nd.quat, i * 4 + 1);
    float y = ld_attr<DT>(nd.quat, i * 4 + 2), z = ld_attr<DT>(nd.quat, i * 4 + 3);
    const float inv = rsqrtf(w * w + x * x + y * y + z * z);
    w *= inv; x *= inv; y *= inv; z *= inv;
    g.r00 = 1.f - 2.f * (y * y + z * z); g.r01 = 2.f * (x * y - w * z); g.r02 = 2.f * (x * z + w * y);
    g.r10 = 2.f * (x * y + w * z); g.r11 = 1.f - 2.f * (x * x + z * z); g.r12 = 2.f * (y * z - w * x);
    g.r20 = 2.f * (x * z - w * y); g.r21 = 2.f * (y * z + w * x); g.r22 = 1.f - 2.f * (x * x + y * y);
    g.smax = fmaxf(g.s0, fmaxf(g.s1, g.s2));
}

struct Splat {
    float u, v, z;
    float a, b, c;        // conic (inverse 2D covariance), used for binning
    float qa, qb, qc;     // q = qa (dx + qb dy)^2 + qc dy^2, used for compositing
    int tx0, tx1, ty0, ty1;
    int x0, x1, y0, y1;   // pixel bounds of the ellipse box, clamped to the image
};

// EWA projection of one Gaussian into one view.  Returns false if culled (near plane,
// degenerate covariance or off screen).
//
// Numerics: with A = J M_R R (2x3) and S = diag(s^2), Sigma2D = A S A^T + lowpass I.  Its
// entries are sums of products with the positive weights s_k^2, and its determinant is
// evaluated by Cauchy-Binet as a sum of positive terms, so thin (flattened) Gaussians do not
// lose their small eigenvalue to cancellation.  The quadratic form is stored factored,
// q = (cyy/det) (dx - (cxy/cyy) dy)^2 + dy^2 / cyy, a sum of two non-negative terms.
__device__ __forceinline__ bool project(const Gauss& g, const VNode& vn, const ViewDesc& vd, const Params& P, Splat& s) {
    const float* M = vn.M;
    // camera-space centre, faithfully rounded (z is the depth key)
    const float z = camera_depth(vn, g.mx, g.my, g.mz);
    if (!(z > P.z_near)) return false;
    const float tx = camera_row(vn, 0, g.mx, g.my, g.mz);
    const float ty = camera_row(vn, 1, g.mx, g.my, g.mz);
    const float iz = 1.f / z;
    const float xr = tx * iz, yr = ty * iz;
    const float xc = fminf(vd.limx, fmaxf(-vd.limx, xr));
    const float yc = fminf(vd.limy, fmaxf(-vd.limy, yr));
    // rows of T = J * M_R:  T0 = fx/z (M_R row0 - xc * M_R row2),  T1 = fy/z (M_R row1 - yc * M_R row2)
    const float fxz = vd.fx * iz, fyz = vd.fy * iz;
    const float t00 = fxz * fmaf(-xc, M[8], M[0]), t01 = fxz * fmaf(-xc, M[9], M[1]), t02 = fxz * fmaf(-xc, M[10], M[2]);
    const float t10 = fyz * fmaf(-yc, M[8], M[4]), t11 = fyz * fmaf(-yc, M[9], M[5]), t12 = fyz * fmaf(-yc, M[10], M[6]);
    // A = T R
    const float a00 = fmaf(t00, g.r00, fmaf(t01, g.r10, t02 * g.r20));
    const float a01 = fmaf(t00, g.r01, fmaf(t01, g.r11, t02 * g.r21));
    const float a02 = fmaf(t00, g.r02, fmaf(t01, g.r12, t02 * g.r22));
    const float a10 = fmaf(t10, g.r00, fmaf(t11, g.r10, t12 * g.r20));
    const float a11 = fmaf(t10, g.r01, fmaf(t11, g.r11, t12 * g.r21));
    const float a12 = fmaf(t10, g.r02, fmaf(t11, g.r12, t12 * g.r22));
    const float sa0 = g.s0 * a00, sa1 = g.s1 * a01, sa2 = g.s2 * a02;
    const float cxx0 = fmaf(sa0, a00, fmaf(sa1, a01, sa2 * a02));
    const float cxy = fmaf(sa0, a10, fmaf(sa1, a11, sa2 * a12));
    const float cyy0 = fmaf(g.s0 * a10, a10, fmaf(g.s1 * a11, a11, g.s2 * a12 * a12));
    const float m01 = fmaf(a00, a11, -a01 * a10), m02 = fmaf(a00, a12, -a02 * a10), m12 = fmaf(a01, a12, -a02 * a11);
    const float det0 = fmaf(g.s0 * g.s1 * m01, m01, fmaf(g.s0 * g.s2 * m02, m02, g.s1 * g.s2 * m12 * m12));
    const float lp = P.lowpass;
    const float cxx = cxx0 + lp, cyy = cyy0 + lp;
    const float det = fmaf(lp, cxx0 + cyy0 + lp, det0);
    if (!(det > 0.f) || !(cyy > 0.f)) return false;
    const float idet = 1.f / det;
    s.a = cyy * idet;
    s.b = -cxy * idet;
    s.c = cxx * idet;
    const float icyy = 1.f / cyy;
    s.qa = s.a;
    s.qb = -cxy * icyy;
    s.qc = icyy;
    s.u = fmaf(vd.fx, xr, vd.cx);
    s.v = fmaf(vd.fy, yr, vd.cy);
    s.z = z;
    // box of {d : d^T conic d <= qbin}: half extents sqrt(qbin * Sigma_ii); pixel centres x + 1/2
    const float hx = sqrtf(P.qbin * cxx), hy = sqrtf(P.qbin * cyy);
    const float fx0 = ceilf(s.u - hx - 0.5f), fx1 = floorf(s.u + hx - 0.5f);
    const float fy0 = ceilf(s.v - hy - 0.5f), fy1 = floorf(s.v + hy - 0.5f);
    if (!(fx1 >= 0.f && fy1 >= 0.f && fx0 <= (float)(vd.W - 1) && fy0 <= (float)(vd.H - 1) && fx0 <= fx1 && fy0 <= fy1))
        return false;
    s.x0 = (int)fmaxf(fx0, 0.f);
    s.x1 = (int)fminf(fx1, (float)(vd.W - 1));
    s.y0 = (int)fmaxf(fy0, 0.f);
    s.y1 = (int)fminf(fy1, (float)(vd.H - 1));
    s.tx0 = s.x0 >> P.tile_sx; s.tx1 = s.x1 >> P.tile_sx;
    s.ty0 = s.y0 >> P.tile_sy; s.ty1 = s.y1 >> P.tile_sy;
    return true;
}

// Conservative screen-space cull and pair bound: 0 only if project() would certainly return
// false; else at least the number of tiles of project()'s pixel box.  The
// 2D covariance satisfies Sigma_xx <= |T0|^2 smax + lowpass with |T0|^2 = (fx/z)^2 (1 + xc^2)
// for the orthonormal rows of camera_from_node, so the ellipse box is bounded by
// sqrt(qbin ((fx/z)^2 (1 + xc^2) smax + lowpass)) (2 % + 1e-3 px of slack for rounding).  The
// camera-space centre is taken from plain FMA chains over the leading parts M; against the
// faithfully rounded centre of project() each coordinate differs by less than 6u S_i (three
// roundings, the omitted trailing parts and the faithful rounding, u = 2^-24, S_i = sum of the
// magnitudes of the row's terms), bounded here by e_i = 2^-20 S_i, which widens the near-plane
// test and the box.  The box, widened to whole pixels and clamped to the image, contains
// project()'s; a centre that may lie at the camera plane counts every tile of the view.
__device__ __forceinline__ uint32_t conservative_tiles(const Gauss& g, const VNode& vn, const ViewDesc& vd,
                                                       const Params& P) {
    const float* M = vn.M;
    const float ax = fabsf(g.mx), ay = fabsf(g.my), az = fabsf(g.mz);
    constexpr float k20 = 9.5367431640625e-07f;   // 2^-20
    const float z = fmaf(M[8], g.mx, fmaf(M[9], g.my, fmaf(M[10], g.mz, M[11])));
    const float ez = k20 * fmaf(fabsf(M[8]), ax, fmaf(fabsf(M[9]), ay, fmaf(fabsf(M[10]), az, fabsf(M[11]))));
    if (!(z + ez > P.z_near)) return 0u;
    const float zl = z - ez;
    if (!(zl > 0.f)) return (uint32_t)(vd.tiles_x * vd.tiles_y);   // at the camera plane: any tile
    const float tx = fmaf(M[0], g.mx, fmaf(M[1], g.my, fmaf(M[2], g.mz, M[3])));
    const float ty = fmaf(M[4], g.mx, fmaf(M[5], g.my, fmaf(M[6], g.mz, M[7])));
    const float ex = k20 * fmaf(fabsf(M[0]), ax, fmaf(fabsf(M[1]), ay, fmaf(fabsf(M[2]), az, fabsf(M[3]))));
    const float ey = k20 * fmaf(fabsf(M[4]), ax, fmaf(fabsf(M[5]), ay, fmaf(fabsf(M[6]), az, fabsf(M[7]))));
    const float iz = 1.f / z;
    const float xr = tx * iz, yr = ty * iz;
    const float xc = fminf(vd.limx, fmaxf(-vd.limx, xr));
    const float yc = fminf(vd.limy, fmaxf(-vd.limy, yr));
    const float fxz = vd.fx * iz, fyz = vd.fy * iz;
    const float s = 1.02f * g.smax;
    // centre error in pixels: |d(t/z)| <= (e_t + |t/z| e_z) / (z - e_z)
    const float izl = 1.f / zl;
    const float dux = vd.fx * fmaf(fabsf(xr), ez, ex) * izl, duy = vd.fy * fmaf(fabsf(yr), ez, ey) * izl;
    const float hx = sqrtf(P.qbin * fmaf(fxz * fxz * fmaf(xc, xc, 1.f), s, P.lowpass)) + 1e-3f + dux;
    const float hy = sqrtf(P.qbin * fmaf(fyz * fyz * fmaf(yc, yc, 1.f), s, P.lowpass)) + 1e-3f + duy;
    const float u = fmaf(vd.fx, xr, vd.cx), v = fmaf(vd.fy, yr, vd.cy);
    const float lx = u - hx - 0.5f, rx = u + hx - 0.5f, ly = v - hy - 0.5f, ry = v + hy - 0.5f;
    if (!(rx >= 0.f && ry >= 0.f && lx <= (float)(vd.W - 1) && ly <= (float)(vd.H - 1))) return 0u;
    const int x0 = (int)fmaxf(floorf(lx), 0.f), x1 = (int)fminf(ceilf(rx), (float)(vd.W - 1));
    const int y0 = (int)fmaxf(floorf(ly), 0.f), y1 = (int)fminf(ceilf(ry), (float)(vd.H - 1));
    return (uint32_t)(((x1 >> P.tile_sx) - (x0 >> P.tile_sx) + 1) * ((y1 >> P.tile_sy) - (y0 >> P.tile_sy) + 1));
}

// Bound of a 32-Gaussian chunk in the node frame: a ball of radius r around c holding every
// mean, and the largest standard deviation sigma.
struct ChunkBound {
    float x, y, z, r, sigma;
};

// Warp-wide: all lanes get the same bound (butterfly sums are bitwise equal on every lane).
// Non-finite values make the bound non-finite, and chunk_may_be_visible then keeps the chunk.
__device__ __forceinline__ ChunkBound chunk_bound(const Gauss& g, bool valid) {
    const uint32_t full = 0xffffffffu;
    const float nv = (float)__popc(__ballot_sync(full, valid));
    float sx = valid ? g.mx : 0.f, sy = valid ? g.my : 0.f, sz = valid ? g.mz : 0.f;
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) {
        sx += __shfl_xor_sync(full, sx, o);
        sy += __shfl_xor_sync(full, sy, o);
        sz += __shfl_xor_sync(full, sz, o);
    }
    ChunkBound b;
    b.x = sx / nv; b.y = sy / nv; b.z = sz / nv;
    const float dx = g.mx - b.x, dy = g.my - b.y, dz = g.mz - b.z;
    const float d = valid ? sqrtf(fmaf(dx, dx, fmaf(dy, dy, dz * dz))) : 0.f;
    const float sg = valid ? sqrtf(g.smax) : 0.f;
    // non-negative floats order like their bit patterns (NaN above +inf)
    b.r = __uint_as_float(__reduce_max_sync(full, __float_as_uint(d)));
    b.sigma = __uint_as_float(__reduce_max_sync(full, __float_as_uint(sg)));
    return b;
}

// Conservative per-view cull of a whole chunk: false only if conservative_tiles() is 0 for
// every Gaussian of the chunk.  conservative_tiles() keeps a Gaussian only if z > z_near and its
// box reaches the image, e.g. u + hx - 1/2 >= 0 on the left, with
//   hx <= k_x (fx / z) sigma + m,   k_x = sqrt(1.02 qbin (1 + limx^2)),  m = sqrt(qbin lowpass) + 1e-3
// (sqrt(a + b) <= sqrt(a) + sqrt(b)).  Multiplied by z > 0 the left condition becomes the
// half-space  fx x + (cx - 1/2 + m) z + k_x fx sigma >= 0  of the camera-space mean, whose
// largest value over the chunk's ball is n.c + |n| r + k_x fx sigma; likewise for the other
// three image edges, and z <= c_z + r for the near plane.  Slack covers the rigid transform's
// orthonormality tolerance (1e-4) and FP32 rounding.
__device__ __forceinline__ bool chunk_may_be_visible(const ChunkBound& b, const VNode& vn, const ViewDesc& vd,
                                                     const Params& P) {
    const float* M = vn.M;
    const float x = fmaf(M[0], b.x, fmaf(M[1], b.y, fmaf(M[2], b.z, M[3])));
    const float y = fmaf(M[4], b.x, fmaf(M[5], b.y, fmaf(M[6], b.z, M[7])));
    const float z = fmaf(M[8], b.x, fmaf(M[9], b.y, fmaf(M[10], b.z, M[11])));
    const float R = fmaf(b.r, 1.001f, 1e-5f * (fabsf(x) + fabsf(y) + fabsf(z)) + 1e-6f);
    if (z + R <= P.z_near) return false;
    const float m = sqrtf(P.qbin * P.lowpass) + 2e-3f;
    const float kx = 1.01f * sqrtf(1.02f * P.qbin * fmaf(vd.limx, vd.limx, 1.f)) * vd.fx * b.sigma;
    const float ky = 1.01f * sqrtf(1.02f * P.qbin * fmaf(vd.limy, vd.limy, 1.f)) * vd.fy * b.sigma;
    const float nzl = vd.cx - 0.5f + m, nzr = (float)vd.W - 0.5f - vd.cx + m;
    const float nzt = vd.cy - 0.5f + m, nzb = (float)vd.H - 0.5f - vd.cy + m;
    // largest value of n.p over the ball, p = (x, y, z) + d, |d| <= R, with a relative slack
    const float fl = fmaf(vd.fx, x, nzl * z) + sqrtf(fmaf(vd.fx, vd.fx, nzl * nzl)) * R + kx;
    const float fr = fmaf(-vd.fx, x, nzr * z) + sqrtf(fmaf(vd.fx, vd.fx, nzr * nzr)) * R + kx;
    const float ft = fmaf(vd.fy, y, nzt * z) + sqrtf(fmaf(vd.fy, vd.fy, nzt * nzt)) * R + ky;
    const float fb = fmaf(-vd.fy, y, nzb * z) + sqrtf(fmaf(vd.fy, vd.fy, nzb * nzb)) * R + ky;
    const float ex = 1e-4f * (vd.fx * fabsf(x) + fmaxf(fabsf(nzl), fabsf(nzr)) * fabsf(z));
    const float ey = 1e-4f * (vd.fy * fabsf(y) + fmaxf(fabsf(nzt), fabsf(nzb)) * fabsf(z));
    return !(fl + ex < 0.f || fr + ex < 0.f || ft + ey < 0.f || fb + ey < 0.f);
}

constexpr int kViewBlock = 8;

struct WarpViews {
    int64_t tab[kViewBlock];      // count-table entry of (view j, chunk)
    uint32_t mask[kViewBlock];    // survivor lanes of view j
    int32_t vv[kViewBlock];       // (view, slot) index of view j, -1 = none
    uint32_t vis[kViewBlock];     // count pass: lanes whose projection succeeded
    uint32_t hits[kViewBlock];    // count pass: tile-rectangle area of view j's visible lanes
    uint32_t ibase[kViewBlock];   // emit: first record of (view j, chunk) relative to the group
};

// ------------------------------------------------------------------ spherical harmonics colour
// Real SH, Condon-Shortley phase, k = l^2 + l + m, for a unit direction (x, y, z):
//   l0: 1/(2 sqrt(pi));  l1: sqrt(3/(4pi)) (-y, z, -x);
//   l2: c2a xy, -c2a yz, c2b (3z^2-1), -c2a xz, c2c (x^2-y^2)
//   l3: -c3a y(3x^2-y^2), c3b xyz, -c3c y(5z^2-1), c3d z(5z^2-3), -c3c x(5z^2-1), c3e z(x^2-y^2),
//       -c3a x(x^2-3y^2)
// with c2a = sqrt(15/(4pi)), c2b = sqrt(5/(16pi)), c2c = sqrt(15/(16pi)), c3a = sqrt(35/(32pi)),
// c3b = sqrt(105/(4pi)), c3c = sqrt(21/(32pi)), c3d = sqrt(7/(16pi)), c3e = sqrt(105/(16pi)).
constexpr float kY00 = 0.28209479177387814f;
constexpr float kC1 = 0.4886025119029199f;
constexpr float kC2a = 1.0925484305920792f, kC2b = 0.31539156525252005f, kC2c = 0.5462742152960396f;
constexpr float kC3a = 0.5900435899266435f, kC3b = 2.890611442640554f, kC3c = 0.4570457994644658f;
constexpr float kC3d = 0.3731763325901154f, kC3e = 1.445305721320277f;

__device__ __forceinline__ void sh_basis(int deg, float x, float y, float z, float Y[16]) {
    Y[0] = kY00;
    if (deg < 1) return;
    Y[1] = -kC1 * y; Y[2] = kC1 * z; Y[3] = -kC1 * x;
    if (deg < 2) return;
    const float xx = x * x, yy = y * y, zz = z * z;
    Y[4] = kC2a * x * y; Y[5] = -kC2a * y * z; Y[6] = kC2b * (3.f * zz - 1.f); Y[7] = -kC2a * x * z;
    Y[8] = kC2c * (xx - yy);
    if (deg < 3) return;
    Y[9] = -kC3a * y * (3.f * xx - yy);
    Y[10] = kC3b * x * y * z;
    Y[11] = -kC3c * y * (5.f * zz - 1.f);
    Y[12] = kC3d * z * (5.f * zz - 3.f);
    Y[13] = -kC3c * x * (5.f * zz - 1.f);
    Y[14] = kC3e * z * (xx - yy);
    Y[15] = -kC3a * x * (xx - 3.f * yy);
}

// Colour of one instance from the warp's staged coefficients (stride kShStride floats per lane).
constexpr int kShStride = 49;   // 48 coefficients + 1 pad: conflict-free lane-strided reads

__device__ __forceinline__ void sh_colour(int deg, const float* __restrict__ coef, const Gauss& g, const VNode& vn,
                                          float rgb[3]) {
    float dx = g.mx - vn.o[0], dy = g.my - vn.o[1], dz = g.mz - vn.o[2];
    const float inv = rsqrtf(dx * dx + dy * dy + dz * dz);
    dx *= inv; dy *= inv; dz *= inv;
    float Y[16];
    sh_basis(deg, dx, dy, dz, Y);
    float r = 0.5f, gg = 0.5f, b = 0.5f;
#pragma unroll
    for (int k = 0; k < 16; ++k) {
        if (k < (deg + 1) * (deg + 1)) {
            r = fmaf(Y[k], coef[k * 3 + 0], r);
            gg = fmaf(Y[k], coef[k * 3 + 1], gg);
            b = fmaf(Y[k], coef[k * 3 + 2], b);
        }
    }
    rgb[0] = fmaxf(r, 0.f); rgb[1] = fmaxf(gg, 0.f); rgb[2] = fmaxf(b, 0.f);
}

// Stages the SH coefficients of the warp's chunk (lane l -> Gaussian chunk*32 + l) as FP32.
template <int DT>
__device__ __forceinline__ void stage_sh(const NodeDesc& nd, int c, int lane, float* __restrict__ sh_smem) {
    const int nc3 = (nd.deg + 1) * (nd.deg + 1) * 3;
    const int64_t g0 = (int64_t)c * kChunk;
    const int cnt = (int)min((int64_t)kChunk, nd.n - g0);
    const int64_t base = g0 * nc3;
    for (int idx = lane; idx < cnt * nc3; idx += 32) {
        const int gl = idx / nc3, k = idx - gl * nc3;
        sh_smem[gl * kShStride + k] = ld_attr<DT>(nd.sh, base + idx);
    }
    __syncwarp();
}

__device__ __forceinline__ int find_node(const NodeDesc* nodes, int n_nodes, int chunk) {
    int lo = 0, hi = n_nodes - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (nodes[mid].chunk0 <= chunk) lo = mid; else hi = mid - 1;
    }
    return lo;
}


// ------------------------------------------------------------------ count and emit passes
// A warp owns a chunk of 32 consecutive Gaussians of one node and walks the (view, slot)
// entries of that node in blocks of kViewBlock views:
//   1. survivors: count pass -- a cull of the whole chunk per view (bounding ball), then a
//      conservative cull of every (lane, view) pair, one ballot per view; emit pass -- the
//      exact visible-lane masks the count pass stored;
//   2. the survivors, queued view-major in Gaussian order, are projected 32 at a time (one
//      per lane);
//   3. count pass -- per view, the mask of lanes whose projection succeeded and the summed
//      area of their tile rectangles (a bound on their tile pairs) go to the count table;
//      emit pass -- record, identity, depth key and exact tile-pair count of each instance at
//      the scanned offset of its (view, chunk) entry.
struct WarpWork {
    WarpViews WV;
    float geo[kChunk * kGeoStride];     // staged geometry of the chunk's Gaussians
};

// Position of the n-th (0-based) set bit of m; requires n < popc(m).
__device__ __forceinline__ int nth_set_bit(uint32_t m, uint32_t n) {
    int pos = 0;
#pragma unroll
    for (int w = 16; w >= 1; w >>= 1) {
        const uint32_t low = __popc(m & ((1u << w) - 1u));
        if (n >= low) { n -= low; m >>= w; pos += w; }
    }
    return pos;
}

// Item `idx` (< total survivors) of a view block: the first view j whose survivors reach past
// idx, and the Gaussian lane g of its (idx - before)-th survivor.
__device__ __forceinline__ void decode_item(uint32_t idx, const WarpViews& WV, int nvb, int& j, int& g) {
    uint32_t before = 0;
    j = 0;
    for (int t = 0; t < nvb; ++t) {
        const uint32_t c = __popc(WV.mask[t]);
        if (idx < before + c) { j = t; break; }
        before += c;
    }
    g = nth_set_bit(WV.mask[j], idx - before);
}

// Outputs of the emit pass, indexed by record (instance) number.
struct EmitOut {
    Record* rec;
    InstInfo* info;
    uint32_t* dkey;       // depth key
    uint32_t* ival;       // the record number itself (value carried by the depth sort)
    uint32_t* ntile;      // tile pairs of the instance
    uint32_t* vig;        // view of the instance within its view group (the depth sort's major key); null: not written
};

template <int DT>
__device__ __forceinline__ void stage_geometry(const NodeDesc& nd, int c, int lane, WarpWork& W, Gauss& g, bool& valid);
template <int DT>
__device__ __forceinline__ void stage_sh(const NodeDesc& nd, int c, int lane, float* __restrict__ sh_smem);

// The emit pass stages the chunk's geometry and SH coefficients at its first visible view
// (lazily: chunks no view sees read nothing but their count-table entries).
template <bool EMIT, int DT>
__device__ __forceinline__ void process_chunk(const NodeDesc& nd, int c, int lane, const NodeView* __restrict__ entries,
                                              int n_entries, int v0, int v1, const ViewDesc* __restrict__ views,
                                              const VNode* __restrict__ vnodes, int K, const Params& P, const Gauss& gme,
                                              bool valid, const ChunkBound& cb, WarpWork& W, float* __restrict__ shc,
                                              uint2* __restrict__ counts, const uint32_t* __restrict__ inst_off,
                                              uint32_t inst_base, const EmitOut& out) {
    WarpViews& WV = W.WV;
    const uint32_t full = 0xffffffffu;
    bool staged = false;
    for (int rb = 0; rb < n_entries; rb += 32) {
        // 1a. a round of 32 views, one per lane.  Count pass: the chunk's bounding ball against
        //     the view (an entry it cannot reach gets its empty count right away); emit pass:
        //     the view's visible-lane mask and record offset from the count table.
        const int e = rb + lane;
        bool keep = false;
        int vv_l = -1;
        int64_t t_l = 0;
        uint32_t m_l = 0, ib_l = 0;
        if (e < n_entries) {
            const NodeView w = entries[e];
            if (w.view >= v0 && w.view < v1) {
                vv_l = w.view * K + w.slot;
                t_l = w.tab + c;
                if constexpr (!EMIT) {
                    keep = chunk_may_be_visible(cb, vnodes[vv_l], views[w.view], P);
                    if (!keep) counts[t_l] = make_uint2(0u, 0u);
                } else {
                    m_l = counts[t_l].x;
                    keep = m_l != 0u;
                    if (keep) ib_l = inst_off[t_l] - inst_base;
                }
            }
        }
        uint32_t surv = __ballot_sync(full, keep);
        if constexpr (EMIT) {
            if (surv && !staged) {
                Gauss gs;
                bool vs;
                stage_geometry<DT>(nd, c, lane, W, gs, vs);
                stage_sh<DT>(nd, c, lane, shc);
                staged = true;
            }
        }
        // 1b. the surviving views, kViewBlock at a time
        while (surv) {
            const int nvb = min(kViewBlock, __popc(surv));
            const int src = nth_set_bit(surv, (uint32_t)min(lane, nvb - 1));
            const int vv_j = __shfl_sync(full, vv_l, src);
            const int64_t t_j = __shfl_sync(full, t_l, src);
            const uint32_t m_j = __shfl_sync(full, m_l, src), ib_j = __shfl_sync(full, ib_l, src);
            if (lane < nvb) {
                WV.vv[lane] = vv_j;
                WV.tab[lane] = t_j;
                WV.vis[lane] = 0;
                WV.hits[lane] = 0;
                WV.mask[lane] = m_j;
                WV.ibase[lane] = ib_j;
            }
            for (int q = 0; q < nvb; ++q) surv &= surv - 1u;   // drop the views taken
            __syncwarp();
            if constexpr (!EMIT) {
                // count pass: the conservative cull decides which instances are emitted and bounds
                // their tile pairs; emission projects them exactly (and writes a dead record for
                // the few, about 2 % on the benchmark batch, that the exact projection rejects)
                for (int j = 0; j < nvb; ++j) {
                    const int vvj = WV.vv[j];
                    const uint32_t a = valid ? conservative_tiles(gme, vnodes[vvj], views[vvj / K], P) : 0u;
                    const uint32_t m = __ballot_sync(full, a != 0u);
                    const uint32_t h = __reduce_add_sync(full, a);
                    if (lane == 0) { WV.mask[j] = m; WV.vis[j] = m; WV.hits[j] = h; }
                }
            }
            __syncwarp();
            uint32_t n_items = 0;
            if constexpr (EMIT)
                for (int j = 0; j < nvb; ++j) n_items += __popc(WV.mask[j]);
            // 2. project the survivors 32 at a time
            for (uint32_t it = 0; it < n_items; it += 32) {
                const uint32_t idx = it + (uint32_t)lane;
                const bool act = idx < n_items;
                int j = 0, g = 0;
                if (act) decode_item(idx, WV, nvb, j, g);
                Splat s;
                bool vis = false;
                Gauss gg;
                const int vvj = act ? WV.vv[j] : 0;
                if (act) {
                    get_geo(W.geo + g * kGeoStride, gg);
                    vis = project(gg, vnodes[vvj], views[vvj / K], P, s);
                }
                if constexpr (EMIT) {
                    uint32_t r = 0;
                    if (act) r = WV.ibase[j] + __popc(WV.mask[j] & ((1u << g) - 1u));
                    const int64_t i = (int64_t)c * kChunk + g;
                    if (act && !vis && in_bounds(r, P.n_rec, P.err, kSiteEmitRecord)) {
                        // kept by the count pass's conservative cull, rejected by the exact
                        // projection: a dead record, last in depth order, with no tile pairs
                        out.rec[r] = Record{};
                        out.info[r] = InstInfo{(uint32_t)(nd.gbase + i), (uint32_t)vvj};
                        out.dkey[r] = (1u << kZBits) - 1u;
                        const uint32_t vg = (uint32_t)vvj / (uint32_t)K - P.view0;
                        out.ival[r] = P.vshift ? r | vg << P.vshift : r;
                        out.ntile[r] = 0u;
                        if (out.vig) out.vig[r] = vg;
                    }
                    if (vis && in_bounds(r, P.n_rec, P.err, kSiteEmitRecord)) {
                        float rgb[3];
                        sh_colour(nd.deg, shc + g * kShStride, gg, vnodes[vvj], rgb);
                        const float op = 1.f / (1.f + __expf(-__ldg(nd.opac + i)));
                        Record R;
                        R.r0 = make_float4(s.u, s.v, op, s.z);
                        R.r1 = make_float4(s.qa, s.qb, s.qc, __uint_as_float((uint32_t)s.x0 | ((uint32_t)s.x1 << 16)));
                        R.r2 = make_float4(rgb[0], rgb[1], rgb[2], __uint_as_float((uint32_t)s.y0 | ((uint32_t)s.y1 << 16)));
                        out.rec[r] = R;
                        out.info[r] = InstInfo{(uint32_t)(nd.gbase + i), (uint32_t)vvj};
                        out.dkey[r] = min(__float_as_uint(s.z) - P.zbase, (1u << kZBits) - 1u);
                        const uint32_t vg = (uint32_t)vvj / (uint32_t)K - P.view0;
                        out.ival[r] = P.vshift ? r | vg << P.vshift : r;
                        if (out.vig) out.vig[r] = vg;
                        // exact tile pairs: the runs of tiles each tile row's band reaches
                        const float4 ext = ellipse_extent(s.qa, s.qb, s.qc, P.qbin);
                        uint32_t npairs = 0;
                        for (int ty = s.ty0; ty <= s.ty1; ++ty) {
                            int t0;
                            npairs += (uint32_t)tile_row_run(s.u, s.v, s.qb, s.qc, ext, s.x0, s.x1, s.y0, s.y1, ty, P, t0);
                        }
                        out.ntile[r] = npairs;
                    }
                }
                __syncwarp();
            }
            // 3. count-table entries of the block
            if constexpr (!EMIT) {
                if (lane < nvb) counts[WV.tab[lane]] = make_uint2(WV.vis[lane], WV.hits[lane]);
            }
            __syncwarp();
        }
    }
}

template <int DT>
__device__ __forceinline__ void stage_geometry(const NodeDesc& nd, int c, int lane, WarpWork& W, Gauss& g, bool& valid) {
    const int64_t i = (int64_t)c * kChunk + lane;
    valid = i < nd.n;
    if (valid) load_geometry<DT>(nd, i, g);
    else { g = Gauss{}; g.s0 = g.s1 = g.s2 = g.smax = 1.f; g.r00 = g.r11 = g.r22 = 1.f; }
    put_geo(W.geo + lane * kGeoStride, g);
    __syncwarp();
}

constexpr int kCountWarps = 4;
constexpr int kEmitWarps = 4;

template <int DT>
__global__ void __launch_bounds__(kCountWarps * 32) k_count_batched(const NodeDesc* __restrict__ nodes, int n_nodes,
        const ViewDesc* __restrict__ views, const VNode* __restrict__ vnodes, int K, const NodeView* __restrict__ nv,
        const int32_t* __restrict__ nv_off, int n_chunks, Params P, int v0, int v1, uint2* counts) {
    __shared__ WarpWork ww[kCountWarps];
    const int chunk = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
    if (chunk >= n_chunks) return;
    const int lane = (int)lane_id();
    WarpWork& W = ww[threadIdx.x >> 5];
    const int k = find_node(nodes, n_nodes, chunk);
    const NodeDesc& nd = nodes[k];
    if (nd.dtype != DT) return;
    const int c = chunk - nd.chunk0;
    Gauss g;
    bool valid;
    stage_geometry<DT>(nd, c, lane, W, g, valid);
    const ChunkBound cb = chunk_bound(g, valid);
    process_chunk<false, DT>(nd, c, lane, nv + nv_off[k], nv_off[k + 1] - nv_off[k], v0, v1, views, vnodes, K, P, g,
                             valid, cb, W, nullptr, counts, nullptr, 0, EmitOut{});
}

// Plain mode: the chunks of one view.  pmap = [K+1 prefix chunk counts in node-id order, K slots].
template <int DT>
__global__ void __launch_bounds__(kCountWarps * 32) k_count_plain(const NodeDesc* __restrict__ nodes,
        const ViewDesc* __restrict__ views, const VNode* __restrict__ vnodes, int K, Params P, int v,
        const int32_t* __restrict__ pmap, int n_view_chunks, uint2* counts) {
    __shared__ WarpWork ww[kCountWarps];
    const int w = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
    if (w >= n_view_chunks) return;
    const int lane = (int)lane_id();
    WarpWork& W = ww[threadIdx.x >> 5];
    int lo = 0, hi = K - 1;
    while (lo < hi) { const int mid = (lo + hi + 1) >> 1; if (pmap[mid] <= w) lo = mid; else hi = mid - 1; }
    const int slot = pmap[K + 1 + lo];
    const NodeDesc& nd = nodes[vnodes[v * K + slot].node];
    if (nd.dtype != DT) return;
    const int c = w - pmap[lo];
    Gauss g;
    bool valid;
    stage_geometry<DT>(nd, c, lane, W, g, valid);
    const ChunkBound cb = chunk_bound(g, valid);
    const NodeView one{v, slot, vnodes[v * K + slot].tab};
    process_chunk<false, DT>(nd, c, lane, &one, 1, v, v + 1, views, vnodes, K, P, g, valid, cb, W, nullptr, counts,
                             nullptr, 0, EmitOut{});
}

template <int DT>
__global__ void __launch_bounds__(kEmitWarps * 32, 5) k_emit_batched(const NodeDesc* __restrict__ nodes, int n_nodes,
        const ViewDesc* __restrict__ views, const VNode* __restrict__ vnodes, int K, const NodeView* __restrict__ nv,
        const int32_t* __restrict__ nv_off, int n_chunks, Params P, int v0, int v1, const uint2* __restrict__ counts,
        const uint32_t* __restrict__ inst_off, uint32_t inst_base, EmitOut out) {
    __shared__ WarpWork ww[kEmitWarps];
    __shared__ float shc[kEmitWarps][kChunk * kShStride];
    const int chunk = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
    if (chunk >= n_chunks) return;
    if (P.gate && *P.gate) return;       // capacity overflow: write nothing
    if (P.inst_base_dev) inst_base = *P.inst_base_dev;
    const int lane = (int)lane_id(), wib = threadIdx.x >> 5;
    WarpWork& W = ww[wib];
    const int k = find_node(nodes, n_nodes, chunk);
    const NodeDesc& nd = nodes[k];
    if (nd.dtype != DT) return;
    const int c = chunk - nd.chunk0;
    process_chunk<true, DT>(nd, c, lane, nv + nv_off[k], nv_off[k + 1] - nv_off[k], v0, v1, views, vnodes, K, P,
                            Gauss{}, false, ChunkBound{}, W, shc[wib], const_cast<uint2*>(counts), inst_off, inst_base,
                            out);
}

template <int DT>
__global__ void __launch_bounds__(kEmitWarps * 32, 5) k_emit_plain(const NodeDesc* __restrict__ nodes,
        const ViewDesc* __restrict__ views, const VNode* __restrict__ vnodes, int K, Params P, int v,
        const int32_t* __restrict__ pmap, int n_view_chunks, const uint2* __restrict__ counts,
        const uint32_t* __restrict__ inst_off, uint32_t inst_base, EmitOut out) {
    __shared__ WarpWork ww[kEmitWarps];
    __shared__ float shc[kEmitWarps][kChunk * kShStride];
    const int w = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
    if (w >= n_view_chunks) return;
    const int lane = (int)lane_id(), wib = threadIdx.x >> 5;
    WarpWork& W = ww[wib];
    int lo = 0, hi = K - 1;
    while (lo < hi) { const int mid = (lo + hi + 1) >> 1; if (pmap[mid] <= w) lo = mid; else hi = mid - 1; }
    const int slot = pmap[K + 1 + lo];
    const NodeDesc& nd = nodes[vnodes[v * K + slot].node];
    if (nd.dtype != DT) return;
    const int c = w - pmap[lo];
    const NodeView one{v, slot, vnodes[v * K + slot].tab};
    process_chunk<true, DT>(nd, c, lane, &one, 1, v, v + 1, views, vnodes, K, P, Gauss{}, false, ChunkBound{}, W,
                            shc[wib], const_cast<uint2*>(counts), inst_off, inst_base, out);
}

// ------------------------------------------------------------------ exclusive scan of the count table
constexpr int kScanThreads = 256, kScanItems = 16, kScanTile = kScanThreads * kScanItems;

__device__ __forceinline__ void block_excl_scan2(uint64_t& a, uint64_t& b, uint64_t& tot_a, uint64_t& tot_b) {
    __shared__ uint64_t sa[kScanThreads / 32], sb[kScanThreads / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    uint64_t xa = a, xb = b;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint64_t ya = __shfl_up_sync(0xffffffffu, xa, o), yb = __shfl_up_sync(0xffffffffu, xb, o);
        if (lane >= o) { xa += ya; xb += yb; }
    }
    if (lane == 31) { sa[wid] = xa; sb[wid] = xb; }
    __syncthreads();
    uint64_t wa = 0, wb = 0;
    tot_a = tot_b = 0;
    for (int w = 0; w < kScanThreads / 32; ++w) {
        if (w < wid) { wa += sa[w]; wb += sb[w]; }
        tot_a += sa[w]; tot_b += sb[w];
    }
    a = wa + xa - a;
    b = wb + xb - b;
    __syncthreads();
}

// The block's kScanTile entries are read warp-striped (coalesced) into shared memory, and each
// thread then takes its kScanItems consecutive entries from there; one pad entry per 16 keeps
// both access patterns free of bank conflicts.
constexpr int kScanPadded = kScanTile + kScanTile / 16;
__device__ __forceinline__ int scan_slot(int k) { return k + (k >> 4); }
__device__ __forceinline__ void load_tile_counts(const uint2* __restrict__ counts, int64_t n, uint2* s_c) {
    const int64_t b0 = (int64_t)blockIdx.x * kScanTile;
#pragma unroll 4
    for (int j = 0; j < kScanItems; ++j) {
        const int k = j * kScanThreads + threadIdx.x;
        s_c[scan_slot(k)] = b0 + k < n ? counts[b0 + k] : make_uint2(0u, 0u);
    }
    __syncthreads();
}

__global__ void __launch_bounds__(kScanThreads) k_scan_partial(const uint2* __restrict__ counts, int64_t n, ulonglong2* parts) {
    __shared__ uint2 s_c[kScanPadded];
    load_tile_counts(counts, n, s_c);
    uint64_t a = 0, b = 0;
    for (int j = 0; j < kScanItems; ++j) {
        const uint2 c = s_c[scan_slot(threadIdx.x * kScanItems + j)];
        a += __popc(c.x); b += c.y;
    }
    uint64_t ta, tb;
    block_excl_scan2(a, b, ta, tb);
    if (threadIdx.x == 0) parts[blockIdx.x] = make_ulonglong2(ta, tb);
}

__global__ void __launch_bounds__(kScanThreads) k_scan_parts(ulonglong2* parts, int64_t n_parts) {
    // single block: exclusive scan of the per-tile totals, in place; parts[n_parts] = grand total
    __shared__ uint64_t carry_a, carry_b;
    if (threadIdx.x == 0) { carry_a = 0; carry_b = 0; }
    __syncthreads();
    for (int64_t base = 0; base < n_parts; base += kScanThreads) {
        const int64_t i = base + threadIdx.x;
        uint64_t a = 0, b = 0;
        if (i < n_parts) { a = parts[i].x; b = parts[i].y; }
        uint64_t ta, tb;
        block_excl_scan2(a, b, ta, tb);
        if (i < n_parts) parts[i] = make_ulonglong2(a + carry_a, b + carry_b);
        __syncthreads();
        if (threadIdx.x == 0) { carry_a += ta; carry_b += tb; }
        __syncthreads();
    }
    if (threadIdx.x == 0) parts[n_parts] = make_ulonglong2(carry_a, carry_b);
}

__global__ void __launch_bounds__(kScanThreads) k_scan_final(const uint2* __restrict__ counts, int64_t n,
                                                            const ulonglong2* __restrict__ parts, uint32_t* inst_off,
                                                            uint64_t* pair_off) {
    __shared__ uint2 s_c[kScanPadded];
    load_tile_counts(counts, n, s_c);
    uint2 c[kScanItems];
    uint64_t a = 0, b = 0;
    for (int j = 0; j < kScanItems; ++j) {
        c[j] = s_c[scan_slot(threadIdx.x * kScanItems + j)];
        a += __popc(c[j].x); b += c[j].y;
    }
    uint64_t ta, tb;
    block_excl_scan2(a, b, ta, tb);
    a += parts[blockIdx.x].x;
    b += parts[blockIdx.x].y;
    // the offsets go back through shared memory so that the stores are warp-striped too; entry
    // n, inside the tile or just past the last one, receives the totals
    const int64_t b0 = (int64_t)blockIdx.x * kScanTile;
    uint64_t* s_p = reinterpret_cast<uint64_t*>(s_c);
    uint32_t* s_i = reinterpret_cast<uint32_t*>(s_c);
    const uint64_t a0 = a;
    __syncthreads();                            // every thread has read its counts
    for (int j = 0; j < kScanItems; ++j) {
        s_p[scan_slot(threadIdx.x * kScanItems + j)] = b;
        b += c[j].y;
    }
    __syncthreads();
#pragma unroll 4
    for (int j = 0; j < kScanItems; ++j) {
        const int k = j * kScanThreads + threadIdx.x;
        if (b0 + k <= n) pair_off[b0 + k] = s_p[scan_slot(k)];
    }
    __syncthreads();
    a = a0;
    for (int j = 0; j < kScanItems; ++j) {
        s_i[scan_slot(threadIdx.x * kScanItems + j)] = (uint32_t)a;
        a += __popc(c[j].x);
    }
    __syncthreads();
#pragma unroll 4
    for (int j = 0; j < kScanItems; ++j) {
        const int k = j * kScanThreads + threadIdx.x;
        if (b0 + k <= n) inst_off[b0 + k] = s_i[scan_slot(k)];
    }
    if (n % kScanTile == 0 && blockIdx.x == gridDim.x - 1 && threadIdx.x == kScanThreads - 1) {
        inst_off[n] = (uint32_t)a; pair_off[n] = b;
    }
}

template <int DT>
void count_launch(const Launch& L, const NodeDesc* nodes, int n_nodes, const ViewDesc* views, const VNode* vnodes, int K,
                  const NodeView* nv, const int32_t* nv_off, int n_chunks, const Params& P, int v0, int v1,
                  bool batched, const int32_t* pmap, int64_t view_chunks, uint2* counts) {
    if (batched) {
        const int blocks = (int)(((int64_t)n_chunks + kCountWarps - 1) / kCountWarps);
        if (blocks == 0) return;
        k_count_batched<DT><<<blocks, kCountWarps * 32, 0, L.stream>>>(nodes, n_nodes, views, vnodes, K, nv, nv_off, n_chunks, P,
                                                          v0, v1, counts);
    } else {
        const int blocks = (int)((view_chunks + kCountWarps - 1) / kCountWarps);
        if (blocks == 0) return;
        k_count_plain<DT><<<blocks, kCountWarps * 32, 0, L.stream>>>(nodes, views, vnodes, K, P, v0, pmap, (int)view_chunks, counts);
    }
    ++*L.launches;
}

template <int DT>
void emit_launch(const Launch& L, const NodeDesc* nodes, int n_nodes, const ViewDesc* views, const VNode* vnodes, int K,
                 const NodeView* nv, const int32_t* nv_off, int n_chunks, const Params& P, int v0, int v1, bool batched,
                 const int32_t* pmap, int64_t view_chunks, const uint2* counts, const uint32_t* inst_off,
                 uint32_t inst_base, const EmitOut& out) {
    if (batched) {
        const int blocks = (int)(((int64_t)n_chunks + kEmitWarps - 1) / kEmitWarps);
        if (blocks == 0) return;
        k_emit_batched<DT><<<blocks, kEmitWarps * 32, 0, L.stream>>>(nodes, n_nodes, views, vnodes, K, nv, nv_off, n_chunks,
                                                                     P, v0, v1, counts, inst_off, inst_base, out);
    } else {
        const int blocks = (int)((view_chunks + kEmitWarps - 1) / kEmitWarps);
        if (blocks == 0) return;
        k_emit_plain<DT><<<blocks, kEmitWarps * 32, 0, L.stream>>>(nodes, views, vnodes, K, P, v0, pmap, (int)view_chunks,
                                                                   counts, inst_off, inst_base, out);
    }
    ++*L.launches;
}

}  // namespace

void launch_setup_views(const Launch& L, const ViewDesc* views, int n_views, const float* node_poses,
                        const int32_t* slot_node, int K, VNode* vnodes, const int64_t* vnode_tab, uint32_t* err) {
    const int n = n_views * K;
    if (n == 0) return;
    k_setup_views<<<(n + 127) / 128, 128, 0, L.stream>>>(views, n_views, node_poses, slot_node, K, vnodes, vnode_tab, err);
    ++*L.launches;
}

void launch_count(const Launch& L, int dtype_mask, const NodeDesc* nodes, int n_nodes, const ViewDesc* views,
                  const VNode* vnodes, int K, const NodeView* node_views, const int32_t* node_view_off,
                  int n_chunks_total, const Params& P, int v0, int v1, bool batched, const int32_t* pmap,
                  int64_t view_chunks, uint2* counts) {
    if (dtype_mask & (1 << DGS_F32))
        count_launch<DGS_F32>(L, nodes, n_nodes, views, vnodes, K, node_views, node_view_off, n_chunks_total, P, v0, v1,
                              batched, pmap, view_chunks, counts);
    if (dtype_mask & (1 << DGS_BF16))
        count_launch<DGS_BF16>(L, nodes, n_nodes, views, vnodes, K, node_views, node_view_off, n_chunks_total, P, v0, v1,
                               batched, pmap, view_chunks, counts);
    if (dtype_mask & (1 << DGS_F16))
        count_launch<DGS_F16>(L, nodes, n_nodes, views, vnodes, K, node_views, node_view_off, n_chunks_total, P, v0, v1,
                              batched, pmap, view_chunks, counts);
}

void launch_emit(const Launch& L, int dtype_mask, const NodeDesc* nodes, int n_nodes, const ViewDesc* views,
                 const VNode* vnodes, int K, const NodeView* node_views, const int32_t* node_view_off,
                 int n_chunks_total, const Params& P, int v0, int v1, bool batched, const int32_t* pmap,
                 int64_t view_chunks, const uint2* counts, const uint32_t* inst_off, uint32_t inst_base,
                 Record* records, InstInfo* info, uint32_t* dkey, uint32_t* ival, uint32_t* ntile, uint32_t* vig) {
    const EmitOut out{records, info, dkey, ival, ntile, vig};
    if (dtype_mask & (1 << DGS_F32))
        emit_launch<DGS_F32>(L, nodes, n_nodes, views, vnodes, K, node_views, node_view_off, n_chunks_total, P, v0, v1,
                             batched, pmap, view_chunks, counts, inst_off, inst_base, out);
    if (dtype_mask & (1 << DGS_BF16))
        emit_launch<DGS_BF16>(L, nodes, n_nodes, views, vnodes, K, node_views, node_view_off, n_chunks_total, P, v0, v1,
                              batched, pmap, view_chunks, counts, inst_off, inst_base, out);
    if (dtype_mask & (1 << DGS_F16))
        emit_launch<DGS_F16>(L, nodes, n_nodes, views, vnodes, K, node_views, node_view_off, n_chunks_total, P, v0, v1,
                             batched, pmap, view_chunks, counts, inst_off, inst_base, out);
}

void launch_scan(const Launch& L, const uint2* counts, int64_t n, uint32_t* inst_off, uint64_t* pair_off,
                 ulonglong2* parts, int64_t n_parts_cap) {
    const int64_t n_parts = (n + kScanTile - 1) / kScanTile;
    (void)n_parts_cap;
    if (n_parts == 0) {
        cudaMemsetAsync(inst_off, 0, sizeof(uint32_t), L.stream);
        cudaMemsetAsync(pair_off, 0, sizeof(uint64_t), L.stream);
        return;
    }
    k_scan_partial<<<(unsigned)n_parts, kScanThreads, 0, L.stream>>>(counts, n, parts);
    k_scan_parts<<<1, kScanThreads, 0, L.stream>>>(parts, n_parts);
    k_scan_final<<<(unsigned)n_parts, kScanThreads, 0, L.stream>>>(counts, n, parts, inst_off, pair_off);
    *L.launches += 3;
}

}  // namespace dgs
