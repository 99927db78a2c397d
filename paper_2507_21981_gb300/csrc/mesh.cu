// Mesh -> Gaussian transfer (Sec. III-B, Mesh-Gaussian Transfer): one flat Gaussian per facet,
// centred on the barycentre, its local frame aligned with the facet's normal and both tangent
// scales equal to the mean barycentre-to-vertex distance.  The normal scale is `flatten` times
// the tangent scale; the opacity logit is an input; the degree-0 SH coefficient comes from the
// mean vertex colour (zero without colours), higher degrees are zero.
//
// One thread per facet: three index loads and three vertex gathers (neighbouring facets share
// vertices, so the gathers mostly hit in cache).  The block stages its facets' means,
// log-scales and colour coefficients in shared memory and writes each output array's
// contiguous range with consecutive threads on consecutive words.  HBM-bound.
#include "dgs_internal.cuh"

namespace dgs {
namespace {

constexpr float kY00 = 0.28209479177387814f;      // real SH basis, degree 0: 1 / (2 sqrt(pi))

__device__ __forceinline__ float3 ld3(const float* p, int64_t i) {
    return make_float3(p[3 * i], p[3 * i + 1], p[3 * i + 2]);
}
__device__ __forceinline__ float3 sub3(float3 a, float3 b) { return make_float3(a.x - b.x, a.y - b.y, a.z - b.z); }
__device__ __forceinline__ float len3(float3 a) { return sqrtf(fmaf(a.x, a.x, fmaf(a.y, a.y, a.z * a.z))); }
__device__ __forceinline__ float3 cross3(float3 a, float3 b) {
    return make_float3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}

constexpr int kMeshThreads = 256;

template <int NC>        // SH coefficients per facet: (degree + 1)^2
__global__ void __launch_bounds__(kMeshThreads) k_mesh_gaussians(const float* __restrict__ v, int64_t n_v, const int32_t* __restrict__ f, int64_t n_f,
                                 const float* __restrict__ col, float flatten, float opacity_logit,
                                 float* __restrict__ o_mean, float* __restrict__ o_ls, float* __restrict__ o_q,
                                 float* __restrict__ o_op, float* __restrict__ o_sh, uint32_t* __restrict__ err) {
    __shared__ float s_mean[kMeshThreads * 3], s_ls[kMeshThreads * 3], s_dc[kMeshThreads * 3];
    const int64_t f0 = (int64_t)blockIdx.x * kMeshThreads;
    const int64_t i = f0 + threadIdx.x;
    const int nb = n_f - f0 < kMeshThreads ? (int)(n_f - f0) : kMeshThreads;   // facets of this block
    if (i < n_f) {
        const int32_t a = f[3 * i], b = f[3 * i + 1], c = f[3 * i + 2];
        float3 bc = make_float3(0.f, 0.f, 0.f);
        float st = 1e-12f, R[3][3] = {{1.f, 0.f, 0.f}, {0.f, 1.f, 0.f}, {0.f, 0.f, 1.f}};
        float3 mc = make_float3(0.5f, 0.5f, 0.5f);
        if (a < 0 || b < 0 || c < 0 || a >= n_v || b >= n_v || c >= n_v) {
            atomicOr(err, kErrIndex);
        } else {
            const float3 p0 = ld3(v, a), p1 = ld3(v, b), p2 = ld3(v, c);
            // everything from the edges, so that a small facet far from the origin keeps its
            // relative accuracy: barycentre p0 + m, m = (e1 + e2) / 3, vertex offsets -m, e1 - m, e2 - m
            const float3 e1 = sub3(p1, p0), e2 = sub3(p2, p0), cr = cross3(e1, e2);
            const float3 m = make_float3((e1.x + e2.x) / 3.f, (e1.y + e2.y) / 3.f, (e1.z + e2.z) / 3.f);
            bc = make_float3(p0.x + m.x, p0.y + m.y, p0.z + m.z);
            st = fmaxf((len3(m) + len3(sub3(e1, m)) + len3(sub3(e2, m))) / 3.f, 1e-12f);
            const float ar = len3(cr), l1 = len3(e1);
            if (ar > 0.f && l1 > 0.f) {
                const float3 n = make_float3(cr.x / ar, cr.y / ar, cr.z / ar);
                const float3 t1 = make_float3(e1.x / l1, e1.y / l1, e1.z / l1);
                const float3 t2 = cross3(n, t1);
                R[0][0] = t1.x; R[1][0] = t1.y; R[2][0] = t1.z;        // columns t1, t2, n
                R[0][1] = t2.x; R[1][1] = t2.y; R[2][1] = t2.z;
                R[0][2] = n.x;  R[1][2] = n.y;  R[2][2] = n.z;
            }
            if (col) {
                const float3 c0 = ld3(col, a), c1 = ld3(col, b), c2 = ld3(col, c);
                mc = make_float3((c0.x + c1.x + c2.x) / 3.f, (c0.y + c1.y + c2.y) / 3.f, (c0.z + c1.z + c2.z) / 3.f);
            }
        }
        // quaternion (w, x, y, z) by Shepperd's method, w >= 0
        const float tr = R[0][0] + R[1][1] + R[2][2];
        float q[4];
        if (tr >= R[0][0] && tr >= R[1][1] && tr >= R[2][2]) {
            const float s = sqrtf(1.f + tr) * 2.f;
            q[0] = 0.25f * s; q[1] = (R[2][1] - R[1][2]) / s; q[2] = (R[0][2] - R[2][0]) / s; q[3] = (R[1][0] - R[0][1]) / s;
        } else if (R[0][0] >= R[1][1] && R[0][0] >= R[2][2]) {
            const float s = sqrtf(1.f + R[0][0] - R[1][1] - R[2][2]) * 2.f;
            q[0] = (R[2][1] - R[1][2]) / s; q[1] = 0.25f * s; q[2] = (R[0][1] + R[1][0]) / s; q[3] = (R[0][2] + R[2][0]) / s;
        } else if (R[1][1] >= R[2][2]) {
            const float s = sqrtf(1.f + R[1][1] - R[0][0] - R[2][2]) * 2.f;
            q[0] = (R[0][2] - R[2][0]) / s; q[1] = (R[0][1] + R[1][0]) / s; q[2] = 0.25f * s; q[3] = (R[1][2] + R[2][1]) / s;
        } else {
            const float s = sqrtf(1.f + R[2][2] - R[0][0] - R[1][1]) * 2.f;
            q[0] = (R[1][0] - R[0][1]) / s; q[1] = (R[0][2] + R[2][0]) / s; q[2] = (R[1][2] + R[2][1]) / s; q[3] = 0.25f * s;
        }
        const float sg = q[0] < 0.f ? -1.f : 1.f;
        const int t3 = 3 * threadIdx.x;
        s_mean[t3] = bc.x; s_mean[t3 + 1] = bc.y; s_mean[t3 + 2] = bc.z;
        const float ls = logf(st);
        s_ls[t3] = ls; s_ls[t3 + 1] = ls; s_ls[t3 + 2] = logf(flatten * st);
        s_dc[t3] = (mc.x - 0.5f) / kY00; s_dc[t3 + 1] = (mc.y - 0.5f) / kY00; s_dc[t3 + 2] = (mc.z - 0.5f) / kY00;
        reinterpret_cast<float4*>(o_q)[i] = make_float4(sg * q[0], sg * q[1], sg * q[2], sg * q[3]);
        o_op[i] = opacity_logit;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < 3 * nb; e += kMeshThreads) {
        o_mean[3 * f0 + e] = s_mean[e];
        o_ls[3 * f0 + e] = s_ls[e];
    }
    constexpr int per = 3 * NC;                        // SH words per facet
    float* sh = o_sh + f0 * per;
    for (int e = threadIdx.x; e < per * nb; e += kMeshThreads) {
        const int fi = e / per, k = e - fi * per;
        sh[e] = k < 3 ? s_dc[3 * fi + k] : 0.f;
    }
}

}  // namespace

void launch_mesh_gaussians(const Launch& L, const float* v, int64_t n_v, const int32_t* f, int64_t n_f,
                           const float* col, float flatten, float opacity_logit, int n_coef, float* mean,
                           float* log_scale, float* quat, float* opac, float* sh, uint32_t* err) {
    if (n_f <= 0) return;
    const unsigned blocks = (unsigned)((n_f + kMeshThreads - 1) / kMeshThreads);
    auto* kern = n_coef == 1 ? k_mesh_gaussians<1> : n_coef == 4 ? k_mesh_gaussians<4>
               : n_coef == 9 ? k_mesh_gaussians<9> : k_mesh_gaussians<16>;
    kern<<<blocks, kMeshThreads, 0, L.stream>>>(v, n_v, f, n_f, col, flatten, opacity_logit, mean, log_scale, quat, opac,
                                                sh, err);
    ++*L.launches;
}

}  // namespace dgs
