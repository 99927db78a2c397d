// LiDAR by Gaussian ray tracing through a per-node BVH (Sec. III-C: LiDAR is simulated by
// native ray tracing of the scene's Gaussians, accelerated by a BVH).
//
// Per ray o + t d (|d| = 1) and Gaussian (mean mu, whitening M = diag(1/s) R^T in its node's
// frame): o' = M (o_n - mu), d' = M d_n; the response peaks at t* = -(o'.d')/(d'.d') with
// Mahalanobis distance q* = |o' x d'|^2 / (d'.d').  A hit needs q* <= q_max and
// r_min <= t* <= r_max; alpha = min(alpha_max, opacity exp(-q*/2)), skipped below alpha_min.
// Hits composite front to back in (t*, global id) order with the camera's termination rule;
// D = sum T alpha t*, A = 1 - T.
//
// Acceleration structure, per node (built once from the node's attributes, in its frame): a
// 64-byte record per Gaussian (mu, opacity, M) and an implicit complete binary tree over
// leaves of 8 consecutive Gaussians in storage order (heap numbering: root 1, children 2k and
// 2k+1, leaves P..2P-1), each node holding the box of the 3-sigma ellipsoids below it.  The
// tree's quality follows the storage order: Z-ordered nodes (dgs_spatial_order) give compact
// leaves.  Trees are never refitted per env: rays are moved into each node's frame instead.
//
// Tracing: one thread per ray, one warp per packet of 32 rays.  A round collects, over every
// node of the ray's env, the K nearest hits whose (t*, id) key follows the last key
// composited, in a sorted buffer in shared memory; the packet's traversal is front to back and skips
// boxes outside every lane's [t_last, t of its K-th hit].  The round's hits are composited;
// the next round resumes after the last of them, until the transmittance drops below t_min or
// fewer than K hits were left.
#include <algorithm>

#include "dgs_internal.cuh"

namespace dgs {
namespace {

constexpr int kLeaf = 8;             // Gaussians per leaf
constexpr int kKbuf = 32;            // hits per round
constexpr int kStack = 40;           // traversal stack (depth <= 31 levels + the far children)
constexpr int kTraceThreads = 128;

__device__ __forceinline__ float sigmoidf(float x) { return 1.f / (1.f + __expf(-x)); }

// Records and leaf boxes of one node: thread i = Gaussian i (threads past n give empty boxes),
// lanes 8j..8j+7 of a warp reduce the box of leaf j.
template <int DT>
__global__ void k_lidar_records(NodeDesc nd, float sq, float4* __restrict__ rec, float4* __restrict__ box,
                                int64_t P) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    if (i < nd.n) {
        const float mx = nd.mean[3 * i], my = nd.mean[3 * i + 1], mz = nd.mean[3 * i + 2];
        float qw = ld_attr<DT>(nd.quat, 4 * i), qx = ld_attr<DT>(nd.quat, 4 * i + 1),
              qy = ld_attr<DT>(nd.quat, 4 * i + 2), qz = ld_attr<DT>(nd.quat, 4 * i + 3);
        const float qn = rsqrtf(qw * qw + qx * qx + qy * qy + qz * qz);
        qw *= qn; qx *= qn; qy *= qn; qz *= qn;
        const float R[3][3] = {{1.f - 2.f * (qy * qy + qz * qz), 2.f * (qx * qy - qw * qz), 2.f * (qx * qz + qw * qy)},
                               {2.f * (qx * qy + qw * qz), 1.f - 2.f * (qx * qx + qz * qz), 2.f * (qy * qz - qw * qx)},
                               {2.f * (qx * qz - qw * qy), 2.f * (qy * qz + qw * qx), 1.f - 2.f * (qx * qx + qy * qy)}};
        float s[3], is[3];
        for (int a = 0; a < 3; ++a) {
            const float l = ld_attr<DT>(nd.log_scale, 3 * i + a);
            s[a] = expf(l);
            is[a] = expf(-l);
        }
        float M[3][3];
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) M[a][b] = R[b][a] * is[a];
        const float op = sigmoidf(nd.opac[i]);
        rec[4 * i + 0] = make_float4(mx, my, mz, op);
        rec[4 * i + 1] = make_float4(M[0][0], M[0][1], M[0][2], M[1][0]);
        rec[4 * i + 2] = make_float4(M[1][1], M[1][2], M[2][0], M[2][1]);
        // squared radius of the sphere holding the q_max ellipsoid: a ray farther from the mean
        // than that cannot hit (cheap test before the exact one)
        const float smax = fmaxf(fmaxf(s[0], s[1]), s[2]);
        rec[4 * i + 3] = make_float4(M[2][2], sq * sq * smax * smax * 1.002f, 0.f, 0.f);
        const float m[3] = {mx, my, mz};
        for (int a = 0; a < 3; ++a) {
            // half extent of the ellipsoid q <= q_max along axis a, widened slightly so that
            // rounding never drops a hit the exact test keeps
            const float h = sq * sqrtf(R[a][0] * R[a][0] * s[0] * s[0] + R[a][1] * R[a][1] * s[1] * s[1] +
                                       R[a][2] * R[a][2] * s[2] * s[2]);
            const float hw = fmaf(h, 1.001f, 1e-6f + 1e-6f * fabsf(m[a]));
            lo[a] = m[a] - hw;
            hi[a] = m[a] + hw;
        }
    }
#pragma unroll
    for (int o = 1; o < kLeaf; o <<= 1) {
        for (int a = 0; a < 3; ++a) {
            lo[a] = fminf(lo[a], __shfl_xor_sync(0xffffffffu, lo[a], o));
            hi[a] = fmaxf(hi[a], __shfl_xor_sync(0xffffffffu, hi[a], o));
        }
    }
    const int64_t leaf = i / kLeaf;
    if ((i & (kLeaf - 1)) == 0 && leaf < P) {
        box[2 * (P + leaf)] = make_float4(lo[0], lo[1], lo[2], 0.f);
        box[2 * (P + leaf) + 1] = make_float4(hi[0], hi[1], hi[2], 0.f);
    }
}

// One tree level of every tree that has it: node k in [h, 2h) = union of its children.
struct LevelJob {
    float4* box;
    int64_t first;           // first thread of this tree in the launch
};

__global__ void k_lidar_level(const LevelJob* __restrict__ jobs, int n_jobs, int64_t h, int64_t total) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= total) return;
    int lo = 0, hi = n_jobs - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (jobs[mid].first <= t) lo = mid; else hi = mid - 1;
    }
    float4* box = jobs[lo].box;
    const int64_t k = h + (t - jobs[lo].first);
    const float4 a0 = box[4 * k], a1 = box[4 * k + 1], b0 = box[4 * k + 2], b1 = box[4 * k + 3];
    box[2 * k] = make_float4(fminf(a0.x, b0.x), fminf(a0.y, b0.y), fminf(a0.z, b0.z), 0.f);
    box[2 * k + 1] = make_float4(fmaxf(a1.x, b1.x), fmaxf(a1.y, b1.y), fmaxf(a1.z, b1.z), 0.f);
}

// Per (sensor, slot): the sensor's rotation and origin expressed in the node's frame.
__global__ void k_lidar_setup(const LidarSensorDev* __restrict__ sensors, int S, const int32_t* __restrict__ slot_node,
                              int K, const float* __restrict__ node_poses, LidarSlot* __restrict__ out,
                              uint32_t* __restrict__ err) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= S * K) return;
    const int s = idx / K, j = idx % K;
    const LidarSensorDev& sd = sensors[s];
    LidarSlot o;
    o.node = slot_node[sd.env * K + j];
    if (o.node >= 0) {
        const float* W = node_poses + ((int64_t)sd.env * K + j) * 12;
        float Wm[12];
        bool ok = true;
        for (int a = 0; a < 12; ++a) {
            Wm[a] = W[a];
            ok &= isfinite(Wm[a]);
        }
        for (int a = 0; a < 3 && ok; ++a)
            for (int b = 0; b < 3; ++b) {
                const float d = Wm[a] * Wm[b] + Wm[4 + a] * Wm[4 + b] + Wm[8 + a] * Wm[8 + b];
                ok &= fabsf(d - (a == b ? 1.f : 0.f)) <= 1e-4f;
            }
        if (!ok) {
            atomicOr(err, kErrPose);
            o.node = -1;
        } else {
            // node_from_sensor = (world_from_node)^-1 world_from_sensor
            const float* P = sd.pose;
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b)
                    o.R[3 * a + b] = Wm[a] * P[b] + Wm[4 + a] * P[4 + b] + Wm[8 + a] * P[8 + b];
            const float v0 = P[3] - Wm[3], v1 = P[7] - Wm[7], v2 = P[11] - Wm[11];
            for (int a = 0; a < 3; ++a) o.o[a] = Wm[a] * v0 + Wm[4 + a] * v1 + Wm[8 + a] * v2;
        }
    }
    out[idx] = o;
}

__device__ __forceinline__ bool slab(const float4 lo, const float4 hi, const float o[3], const float id[3], float t_lo,
                                     float t_hi) {
    if (lo.x > hi.x) return false;                   // empty box
    const float x0 = (lo.x - o[0]) * id[0], x1 = (hi.x - o[0]) * id[0];
    const float y0 = (lo.y - o[1]) * id[1], y1 = (hi.y - o[1]) * id[1];
    const float z0 = (lo.z - o[2]) * id[2], z1 = (hi.z - o[2]) * id[2];
    // fminf/fmaxf drop the NaN of 0 * inf (ray parallel to a slab through its origin)
    const float enter = fmaxf(fmaxf(fminf(x0, x1), fminf(y0, y1)), fmaxf(fminf(z0, z1), t_lo));
    const float exit = fminf(fminf(fmaxf(x0, x1), fmaxf(y0, y1)), fminf(fmaxf(z0, z1), t_hi));
    return enter <= exit;
}

__device__ __forceinline__ float slab_enter(const float4 lo, const float4 hi, const float o[3], const float id[3]) {
    const float x0 = (lo.x - o[0]) * id[0], x1 = (hi.x - o[0]) * id[0];
    const float y0 = (lo.y - o[1]) * id[1], y1 = (hi.y - o[1]) * id[1];
    const float z0 = (lo.z - o[2]) * id[2], z1 = (hi.z - o[2]) * id[2];
    return fmaxf(fmaxf(fminf(x0, x1), fminf(y0, y1)), fminf(z0, z1));
}

// Per lane, in dynamic shared memory (lane-interleaved: entry i of thread x at [i][x]): the
// round's sorted hits as bits of t*, global id and alpha; (t bits, id) is the 64-bit order key.
constexpr size_t kKbufBytes = (size_t)3 * kKbuf * kTraceThreads * sizeof(uint32_t);

// Warp = a packet of up to 32 rays (consecutive ray numbers: make them neighbours in the beam
// pattern).  The packet walks each tree together on a warp-uniform stack: a box is descended
// if it holds the interval of any lane's ray, the children in the order of the first such
// lane's entry distances; records and boxes are read once per warp.  Each lane keeps its own
// hit buffer, interval and compositing state, and rounds repeat while any lane is unfinished.
// Lanes whose sensor differs in a slot's node take the tree in turns.  Warps are persistent:
// each takes the next 32 rays from a counter until none are left, so that packets of very
// different cost (rays grazing a surface, many rounds) do not leave SMs idle at the end.
__global__ void __launch_bounds__(kTraceThreads) k_lidar_trace(const LidarTreeDev* __restrict__ trees,
                                                               const LidarSlot* __restrict__ slots, int K,
                                                               const float* __restrict__ dirs, int n_dirs,
                                                               int64_t n_rays, LidarParams LP,
                                                               float* __restrict__ out_d, float* __restrict__ out_a,
                                                               uint32_t* __restrict__ err,
                                                               unsigned long long* __restrict__ next_ray,
                                                               unsigned long long n_packets, unsigned long long scramble) {
    __shared__ int s_stack[kTraceThreads / 32][kStack];
    extern __shared__ uint32_t s_kbuf[];
    uint32_t* const kt = s_kbuf + threadIdx.x;                      // entry i at kt[i * kTraceThreads]
    uint32_t* const kg = kt + kKbuf * kTraceThreads;
    float* const ka = reinterpret_cast<float*>(kg + kKbuf * kTraceThreads);
    const int lane = threadIdx.x & 31;
    int* stk = s_stack[threadIdx.x >> 5];
    for (;;) {
        unsigned long long pk = 0;
        if (lane == 0) pk = atomicAdd(next_ray, 1ull);
        pk = __shfl_sync(0xffffffffu, pk, 0);
        if (pk >= n_packets) break;
        // packets in a scrambled order (p -> p * scramble mod n_packets, a bijection): costly
        // packets that are neighbours in ray order do not all start last
        const unsigned long long base = (unsigned long long)((unsigned __int128)pk * scramble % n_packets) * 32ull;
        const int64_t ray = (int64_t)base + lane;
        const bool valid = ray < n_rays;
        int s = 0, j = 0;
        float ds[3] = {1.f, 0.f, 0.f};
        if (valid) {
            s = (int)(ray / n_dirs);
            j = (int)(ray - (int64_t)s * n_dirs);
            ds[0] = dirs[3 * j]; ds[1] = dirs[3 * j + 1]; ds[2] = dirs[3 * j + 2];
            const float r = rsqrtf(ds[0] * ds[0] + ds[1] * ds[1] + ds[2] * ds[2]);
            ds[0] *= r; ds[1] *= r; ds[2] *= r;
        }
        const LidarSlot* sl = slots + (int64_t)s * K;
        float T = 1.f, D = 0.f;
        uint64_t last = 0;                                 // keys <= last are composited
        bool first = true, done = !valid;
        while (__any_sync(0xffffffffu, !done)) {
            int cnt = 0;
            uint64_t maxkey = ~0ull;                   // key of the last entry once the buffer is full
            const float t_lo = first ? LP.r_min : __uint_as_float((uint32_t)(last >> 32));
            float t_hi = LP.r_max;
            for (int slot = 0; slot < K; ++slot) {
                int my_node = -1;
                float o[3] = {0.f, 0.f, 0.f}, d[3] = {1.f, 1.f, 1.f}, id[3] = {1.f, 1.f, 1.f};
                if (!done) {
                    const LidarSlot& S = sl[slot];
                    my_node = S.node;
                    if (my_node >= 0 && trees[my_node].n == 0) my_node = -1;
                    if (my_node >= 0) {
                        for (int a = 0; a < 3; ++a) {
                            o[a] = S.o[a];
                            d[a] = S.R[3 * a] * ds[0] + S.R[3 * a + 1] * ds[1] + S.R[3 * a + 2] * ds[2];
                            id[a] = 1.f / d[a];
                        }
                    }
                }
                unsigned pending = __ballot_sync(0xffffffffu, my_node >= 0);
                while (pending) {
                    const int node = __shfl_sync(0xffffffffu, my_node, __ffs(pending) - 1);
                    const unsigned mine_mask = __ballot_sync(0xffffffffu, my_node == node) & pending;
                    pending &= ~mine_mask;
                    const bool mine = (mine_mask >> lane) & 1u;
                    const LidarTreeDev tr = trees[node];
                    int sp = 0;
                    if (__any_sync(0xffffffffu, mine && slab(tr.box[2], tr.box[3], o, id, t_lo, t_hi))) {
                        if (lane == 0) stk[0] = 1;
                        sp = 1;
                    }
                    __syncwarp();
                    while (sp > 0) {
                        const int64_t k = stk[--sp];
                        __syncwarp();                        // every lane has read before lane 0 writes
                        if (k >= tr.P) {
                            const int64_t g0 = (k - tr.P) * kLeaf;
                            const int64_t g1 = min(g0 + kLeaf, tr.n);
                            // the next Gaussian's record is loaded while this one is tested
                            float4 n0 = make_float4(0.f, 0.f, 0.f, 0.f), n1 = n0, n2 = n0, n3 = n0;
                            if (g0 < g1) {
                                n0 = __ldg(tr.rec + 4 * g0); n1 = __ldg(tr.rec + 4 * g0 + 1);
                                n2 = __ldg(tr.rec + 4 * g0 + 2); n3 = __ldg(tr.rec + 4 * g0 + 3);
                            }
                            for (int64_t g = g0; g < g1; ++g) {
                                const float4 r0 = n0, r1 = n1, r2 = n2, r3 = n3;
                                if (g + 1 < g1) {
                                    n0 = __ldg(tr.rec + 4 * (g + 1)); n1 = __ldg(tr.rec + 4 * (g + 1) + 1);
                                    n2 = __ldg(tr.rec + 4 * (g + 1) + 2); n3 = __ldg(tr.rec + 4 * (g + 1) + 3);
                                }
                                if (!mine) continue;
                                const float v0 = o[0] - r0.x, v1 = o[1] - r0.y, v2 = o[2] - r0.z;
                                {
                                    const float x0 = fmaf(v1, d[2], -v2 * d[1]), x1 = fmaf(v2, d[0], -v0 * d[2]),
                                                x2 = fmaf(v0, d[1], -v1 * d[0]);
                                    if (fmaf(x0, x0, fmaf(x1, x1, x2 * x2)) > r3.y) continue;   // |d| = 1 up to rounding
                                }
                                const float op0 = fmaf(r1.x, v0, fmaf(r1.y, v1, r1.z * v2));
                                const float op1 = fmaf(r1.w, v0, fmaf(r2.x, v1, r2.y * v2));
                                const float op2 = fmaf(r2.z, v0, fmaf(r2.w, v1, r3.x * v2));
                                const float dp0 = fmaf(r1.x, d[0], fmaf(r1.y, d[1], r1.z * d[2]));
                                const float dp1 = fmaf(r1.w, d[0], fmaf(r2.x, d[1], r2.y * d[2]));
                                const float dp2 = fmaf(r2.z, d[0], fmaf(r2.w, d[1], r3.x * d[2]));
                                const float dd = fmaf(dp0, dp0, fmaf(dp1, dp1, dp2 * dp2));
                                const float od = fmaf(op0, dp0, fmaf(op1, dp1, op2 * dp2));
                                const float c0 = fmaf(op1, dp2, -op2 * dp1), c1 = fmaf(op2, dp0, -op0 * dp2),
                                            c2 = fmaf(op0, dp1, -op1 * dp0);
                                const float idd = 1.f / dd;
                                const float t = -od * idd;
                                const float q = fmaf(c0, c0, fmaf(c1, c1, c2 * c2)) * idd;
                                if (!(q <= LP.q_max) || !(t >= LP.r_min) || !(t <= LP.r_max)) continue;
                                const uint64_t key = ((uint64_t)__float_as_uint(t) << 32) | (uint32_t)(tr.gbase + g);
                                if ((!first && key <= last) || key >= maxkey) continue;
                                const float alpha = fminf(LP.alpha_max, r0.w * fast_exp2(kHalfLog2e * q));
                                if (alpha < LP.alpha_min) continue;
                                // insert in order; a full buffer drops its last entry
                                int i = cnt < kKbuf ? cnt : kKbuf - 1;
                                while (i > 0) {
                                    const uint32_t pt = kt[(i - 1) * kTraceThreads], pg = kg[(i - 1) * kTraceThreads];
                                    if ((((uint64_t)pt << 32) | pg) < key) break;
                                    kt[i * kTraceThreads] = pt;
                                    kg[i * kTraceThreads] = pg;
                                    ka[i * kTraceThreads] = ka[(i - 1) * kTraceThreads];
                                    --i;
                                }
                                kt[i * kTraceThreads] = (uint32_t)(key >> 32);
                                kg[i * kTraceThreads] = (uint32_t)key;
                                ka[i * kTraceThreads] = alpha;
                                if (cnt < kKbuf) ++cnt;
                                if (cnt == kKbuf) {
                                    const uint32_t lt = kt[(kKbuf - 1) * kTraceThreads];
                                    maxkey = ((uint64_t)lt << 32) | kg[(kKbuf - 1) * kTraceThreads];
                                    t_hi = __uint_as_float(lt);
                                }
                            }
                        } else {
                            const int64_t c = 2 * k;
                            const float4 l0 = __ldg(tr.box + 2 * c), h0 = __ldg(tr.box + 2 * c + 1),
                                         l1 = __ldg(tr.box + 2 * c + 2), h1 = __ldg(tr.box + 2 * c + 3);
                            const bool in0 = mine && slab(l0, h0, o, id, t_lo, t_hi);
                            const bool in1 = mine && slab(l1, h1, o, id, t_lo, t_hi);
                            const unsigned b0 = __ballot_sync(0xffffffffu, in0), b1 = __ballot_sync(0xffffffffu, in1);
                            if (b0 && b1) {
                                const bool near0 = slab_enter(l0, h0, o, id) <= slab_enter(l1, h1, o, id);
                                const bool n0 = __shfl_sync(0xffffffffu, near0, __ffs(b0 | b1) - 1);
                                if (sp + 2 > kStack) {
                                    if (lane == 0) atomicOr(err, kErrCapacity);
                                    break;
                                }
                                if (lane == 0) {
                                    stk[sp] = (int)(n0 ? c + 1 : c);     // far child below, near on top
                                    stk[sp + 1] = (int)(n0 ? c : c + 1);
                                }
                                sp += 2;
                            } else if (b0 || b1) {
                                if (sp + 1 > kStack) {
                                    if (lane == 0) atomicOr(err, kErrCapacity);
                                    break;
                                }
                                if (lane == 0) stk[sp] = (int)(b0 ? c : c + 1);
                                sp += 1;
                            }
                            __syncwarp();
                        }
                    }
                    __syncwarp();
                }
            }
            if (!done) {
                // composite this round's hits in order
                for (int i = 0; i < cnt && !done; ++i) {
                    const float a = ka[i * kTraceThreads];
                    const float Tn = fmaf(-a, T, T);
                    if (Tn < LP.t_min) {
                        done = true;
                    } else {
                        D = fmaf(a * T, __uint_as_float(kt[i * kTraceThreads]), D);
                        T = Tn;
                    }
                }
                if (cnt < kKbuf) done = true;
                last = maxkey;
                first = false;
            }
        }
        if (valid) {
            out_d[ray] = D;
            out_a[ray] = 1.f - T;
        }
    }
}

}  // namespace

size_t lidar_tree_nodes(int64_t n) {
    if (n <= 0) return 0;
    const int64_t leaves = (n + kLeaf - 1) / kLeaf;
    int64_t P = 1;
    while (P < leaves) P <<= 1;
    return (size_t)(2 * P);
}

void launch_lidar_records(const Launch& L, const NodeDesc& nd, float q_max, float4* rec, float4* box, int64_t P) {
    if (nd.n <= 0) return;
    const int64_t threads = P * kLeaf;              // every leaf, padding leaves included
    const unsigned blocks = (unsigned)((threads + 255) / 256);
    const float sq = sqrtf(q_max);
    switch (nd.dtype) {
        case DGS_BF16: k_lidar_records<DGS_BF16><<<blocks, 256, 0, L.stream>>>(nd, sq, rec, box, P); break;
        case DGS_F16: k_lidar_records<DGS_F16><<<blocks, 256, 0, L.stream>>>(nd, sq, rec, box, P); break;
        default: k_lidar_records<DGS_F32><<<blocks, 256, 0, L.stream>>>(nd, sq, rec, box, P); break;
    }
    ++*L.launches;
}

void launch_lidar_level(const Launch& L, const void* jobs, int n_jobs, int64_t h, int64_t total) {
    if (total <= 0) return;
    k_lidar_level<<<(unsigned)((total + 255) / 256), 256, 0, L.stream>>>(static_cast<const LevelJob*>(jobs), n_jobs,
                                                                           h, total);
    ++*L.launches;
}

size_t lidar_level_job_bytes() { return sizeof(LevelJob); }

void lidar_level_job(void* jobs, int i, float4* box, int64_t first) {
    static_cast<LevelJob*>(jobs)[i] = LevelJob{box, first};
}

void launch_lidar_setup(const Launch& L, const LidarSensorDev* sensors, int S, const int32_t* slot_node, int K,
                        const float* node_poses, LidarSlot* out, uint32_t* err) {
    const int n = S * K;
    if (n == 0) return;
    k_lidar_setup<<<(n + 127) / 128, 128, 0, L.stream>>>(sensors, S, slot_node, K, node_poses, out, err);
    ++*L.launches;
}

void launch_lidar_trace(const Launch& L, const LidarTreeDev* trees, const LidarSlot* slots, int K, const float* dirs,
                        int n_dirs, int64_t n_rays, const LidarParams& LP, float* out_d, float* out_a, uint32_t* err,
                        unsigned long long* next_ray) {
    if (n_rays <= 0) return;
    static int resident = 0, sms = 0;           // blocks per SM at this kernel's resources
    if (!resident) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaFuncSetAttribute(k_lidar_trace, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kKbufBytes);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&resident, k_lidar_trace, kTraceThreads, kKbufBytes);
        resident = std::max(resident, 1);
    }
    const int64_t need = (n_rays + kTraceThreads - 1) / kTraceThreads;
    const unsigned blocks = (unsigned)std::min<int64_t>(need, (int64_t)resident * sms);
    const unsigned long long n_packets = (unsigned long long)(n_rays + 31) / 32;
    unsigned long long a = 0x9E3779B97F4A7C15ull % n_packets;          // a multiplier coprime with n_packets
    auto gcd = [](unsigned long long x, unsigned long long y) { while (y) { const auto t = x % y; x = y; y = t; } return x; };
    if (a == 0) a = 1;
    while (gcd(a, n_packets) != 1) ++a;
    k_lidar_trace<<<blocks, kTraceThreads, kKbufBytes, L.stream>>>(trees, slots, K, dirs, n_dirs, n_rays, LP, out_d,
                                                                   out_a, err, next_ray, n_packets, a);
    ++*L.launches;
}

}  // namespace dgs
