// FP64 CPU oracle of LiDAR simulation by Gaussian ray tracing.
//
// TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or call this file: it
// lets tests/ and the benchmark's CPU-baseline leg check and time the CUDA tracer against a
// slow, obviously correct definition.  It shares no code with the CUDA library.
//
// Sec. III-C: LiDAR is rendered by native ray tracing of the same Gaussian primitives that the
// cameras splat, accelerated by a BVH (the paper gives no further detail).  The definition
// taken here, for one ray x(t) = o + t d (|d| = 1, t in metres) through the Gaussians of every
// node present in the sensor's env:
//   * Gaussian i (node frame mean mu, rotation R from the normalised quaternion, standard
//     deviations s = exp(log_scale), opacity sigmoid(logit)) is transformed with its node's
//     world_from_node pose; in its whitened frame, M = diag(1/s) R^T, the ray is
//     o' = M (o_n - mu) + t M d_n and the Mahalanobis distance q(t) = |o' + t d'|^2 is least at
//       t* = -(o'.d') / (d'.d'),   q* = |o' x d'|^2 / (d'.d')
//     (the point of the ray where the Gaussian's density peaks).
//   * The ray hits Gaussian i iff q* <= q_max (the 3-sigma ellipsoid) and r_min <= t* <= r_max;
//     its opacity along the ray is alpha = min(alpha_max, opacity * exp(-q*/2)), skipped when
//     alpha < alpha_min.
//   * Hits are composited in order of (t*, global id), global id = node_base + index:
//     T_next = T (1 - alpha), stop without compositing once T_next < t_min;
//     D = sum T alpha t* (not normalised), A = 1 - T_final.  The range of the return is D / A.
// The oracle tests every Gaussian of every node in the env (no acceleration structure).
//
// Tolerance.  The GPU evaluates the same quantities in binary32.  With u = 2^-24, m the
// largest whitening gain max 1/s and L = |o_n| + |mu| + |t_node| + |t_sensor| + 1 (metres):
//   e_o = 6 u m L                    absolute error of o' (pose composition, subtraction, M)
//   e_d = 6 u m                      absolute error of d'
//   e_p = e_o + |o'| e_d / |d'|      error of the part of o' normal to d'
//   e_q = 2 sqrt(q*) e_p + e_p^2 + 8 u q*,   e_t = e_p / |d'| + 8 u (|t*| + L)
//   e_alpha = alpha (e_q / 2 + 2^-20)
// A decision is ambiguous when its quantity lies within twice its error of the threshold (plus
// eps_rel relative): the ellipsoid (q*), the range window (t*), alpha_min, and the termination
// (T_next against t_min, with e_T = T_next (sum alpha/(1-alpha) e_alpha/alpha + 2u k)).  The
// oracle composites the primary branch and returns per ray a tolerance on D and A that adds
//   - the continuous errors: sum T e_alpha on A; sum w (e_t + t* e_alpha/alpha) + 4u k D on D;
//   - per ambiguous inclusion of hit k (T_k = transmittance in front of it): alpha_k T_k on A,
//     alpha_k (T_k t*_k + D_behind / (1 - alpha_k)) on D (removing or adding one factor
//     (1 - alpha_k) rescales everything behind it);
//   - per ambiguous termination at hit k: T_k on A and T_k t_far on D (all that could follow);
//   - per pair of neighbours in the order whose t* differ by less than their errors:
//     (w_i + w_j) |t*_i - t*_j| + 2 (e_t,i + e_t,j)(w_i + w_j) on D.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdint>
#include <thread>
#include <vector>

extern "C" {

typedef struct {
    int32_t n_nodes;
    const int64_t* node_n;         // [n_nodes]
    const double* mean;            // [G,3] node-major
    const double* log_scale;       // [G,3]
    const double* quat;            // [G,4] (w,x,y,z)
    const double* opacity_logit;   // [G]
    int32_t E, K;
    const int32_t* env_node_ids;   // [E,K] -1 = empty
    const double* node_poses;      // [E,K,12] world_from_node
} oracle_lidar_scene;

typedef struct {
    double alpha_min, alpha_max, t_min, q_max, r_min, r_max, eps_rel;
    int32_t nthreads;
} oracle_lidar_opts;

}  // extern "C"

namespace {

constexpr double kU = 1.0 / 16777216.0;   // 2^-24

struct Hit {
    double t, alpha, e_t, e_alpha;
    int64_t gid;
    bool amb;          // inclusion decision ambiguous
};

struct NodeGeo {       // per Gaussian: whitening and extent, in the node frame
    double mu[3], M[3][3], opac, m;
};

void rot_from_quat(const double q0[4], double R[3][3]) {
    const double n = std::sqrt(q0[0] * q0[0] + q0[1] * q0[1] + q0[2] * q0[2] + q0[3] * q0[3]);
    const double w = q0[0] / n, x = q0[1] / n, y = q0[2] / n, z = q0[3] / n;
    R[0][0] = 1 - 2 * (y * y + z * z); R[0][1] = 2 * (x * y - w * z); R[0][2] = 2 * (x * z + w * y);
    R[1][0] = 2 * (x * y + w * z); R[1][1] = 1 - 2 * (x * x + z * z); R[1][2] = 2 * (y * z - w * x);
    R[2][0] = 2 * (x * z - w * y); R[2][1] = 2 * (y * z + w * x); R[2][2] = 1 - 2 * (x * x + y * y);
}

double norm3(const double v[3]) { return std::sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]); }

template <class F>
void parallel_for(int64_t n, int nth, F&& f) {
    if (n <= 0) return;
    std::atomic<int64_t> next(0);
    auto worker = [&]() {
        for (;;) {
            const int64_t i = next.fetch_add(1);
            if (i >= n) break;
            f(i);
        }
    };
    nth = (int)std::max<int64_t>(1, std::min<int64_t>(nth, n));
    std::vector<std::thread> ts;
    for (int t = 1; t < nth; ++t) ts.emplace_back(worker);
    worker();
    for (auto& t : ts) t.join();
}

}  // namespace

extern "C" {

// Sec. III-C (LiDAR by ray tracing the Gaussians): traces rays (sensor s, direction j) for
// s < n_sensors, j < n_dirs.
//   sensor_env[S], sensor_pose[S,12] (world_from_sensor), dirs[J,3] (sensor frame, normalised here)
//   outputs [S,J]: D, A, their tolerances, hits composited, ambiguous decisions seen
int oracle_lidar_rays(const oracle_lidar_scene* sc, const oracle_lidar_opts* o, int32_t n_sensors,
                      const int32_t* sensor_env, const double* sensor_pose, int32_t n_dirs, const double* dirs,
                      double* out_d, double* out_a, double* tol_d, double* tol_a, int32_t* n_comp, int32_t* n_amb) {
    // per-Gaussian geometry, node by node
    std::vector<int64_t> base(sc->n_nodes + 1, 0);
    for (int k = 0; k < sc->n_nodes; ++k) base[k + 1] = base[k] + sc->node_n[k];
    std::vector<NodeGeo> geo((size_t)base[sc->n_nodes]);
    for (int64_t g = 0; g < base[sc->n_nodes]; ++g) {
        NodeGeo& G = geo[g];
        double R[3][3];
        rot_from_quat(sc->quat + 4 * g, R);
        double inv_s[3];
        for (int a = 0; a < 3; ++a) inv_s[a] = std::exp(-sc->log_scale[3 * g + a]);
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) G.M[a][b] = inv_s[a] * R[b][a];
        for (int a = 0; a < 3; ++a) G.mu[a] = sc->mean[3 * g + a];
        G.opac = 1.0 / (1.0 + std::exp(-sc->opacity_logit[g]));
        G.m = std::max(inv_s[0], std::max(inv_s[1], inv_s[2]));
    }
    const int nth = o->nthreads > 0 ? o->nthreads : std::max(1u, std::thread::hardware_concurrency());
    const int64_t n_rays = (int64_t)n_sensors * n_dirs;
    parallel_for(n_rays, nth, [&](int64_t ray) {
        const int s = (int)(ray / n_dirs), j = (int)(ray % n_dirs);
        const int e = sensor_env[s];
        const double* P = sensor_pose + 12 * s;
        double ds[3] = {dirs[3 * j], dirs[3 * j + 1], dirs[3 * j + 2]};
        const double dn = norm3(ds);
        for (double& v : ds) v /= dn;
        const double ow[3] = {P[3], P[7], P[11]};
        double dw[3];
        for (int a = 0; a < 3; ++a) dw[a] = P[4 * a] * ds[0] + P[4 * a + 1] * ds[1] + P[4 * a + 2] * ds[2];
        std::vector<Hit> hits;
        std::vector<Hit> amb_out;       // ambiguous candidates left out of the primary branch
        for (int slot = 0; slot < sc->K; ++slot) {
            const int k = sc->env_node_ids[e * sc->K + slot];
            if (k < 0) continue;
            const double* W = sc->node_poses + 12 * ((int64_t)e * sc->K + slot);
            // node frame: o_n = R^T (o - t), d_n = R^T d
            double on[3], dnn[3];
            for (int a = 0; a < 3; ++a) {
                on[a] = W[a] * (ow[0] - W[3]) + W[4 + a] * (ow[1] - W[7]) + W[8 + a] * (ow[2] - W[11]);
                dnn[a] = W[a] * dw[0] + W[4 + a] * dw[1] + W[8 + a] * dw[2];
            }
            const double tnode[3] = {W[3], W[7], W[11]};
            const double L0 = norm3(on) + norm3(tnode) + norm3(ow) + 1.0;
            for (int64_t i = 0; i < sc->node_n[k]; ++i) {
                const int64_t g = base[k] + i;
                const NodeGeo& G = geo[g];
                double v[3] = {on[0] - G.mu[0], on[1] - G.mu[1], on[2] - G.mu[2]};
                double op[3], dp[3];
                for (int a = 0; a < 3; ++a) {
                    op[a] = G.M[a][0] * v[0] + G.M[a][1] * v[1] + G.M[a][2] * v[2];
                    dp[a] = G.M[a][0] * dnn[0] + G.M[a][1] * dnn[1] + G.M[a][2] * dnn[2];
                }
                const double dd = dp[0] * dp[0] + dp[1] * dp[1] + dp[2] * dp[2];
                const double od = op[0] * dp[0] + op[1] * dp[1] + op[2] * dp[2];
                const double cx = op[1] * dp[2] - op[2] * dp[1], cy = op[2] * dp[0] - op[0] * dp[2],
                             cz = op[0] * dp[1] - op[1] * dp[0];
                const double t = -od / dd, q = (cx * cx + cy * cy + cz * cz) / dd;
                // FP32 error model (file header)
                const double L = L0 + norm3(G.mu);
                const double e_o = 6 * kU * G.m * L, e_d = 6 * kU * G.m;
                const double nd = std::sqrt(dd), no = norm3(op);
                const double e_p = e_o + no * e_d / nd;
                const double e_q = 2 * std::sqrt(q) * e_p + e_p * e_p + 8 * kU * q + o->eps_rel * o->q_max;
                const double e_t = e_p / nd + 8 * kU * (std::fabs(t) + L) + o->eps_rel * std::fabs(t);
                const bool q_in = q <= o->q_max, q_amb = std::fabs(q - o->q_max) <= 2 * e_q;
                const bool t_in = t >= o->r_min && t <= o->r_max;
                const bool t_amb = std::fabs(t - o->r_min) <= 2 * e_t || std::fabs(t - o->r_max) <= 2 * e_t;
                if (!(q_in || q_amb) || !(t_in || t_amb)) continue;
                const double alpha = std::min(o->alpha_max, G.opac * std::exp(-0.5 * q));
                const double e_alpha = alpha * (0.5 * e_q + 1.0 / 1048576.0) + o->eps_rel * alpha;
                const bool a_in = alpha >= o->alpha_min, a_amb = std::fabs(alpha - o->alpha_min) <= 2 * e_alpha;
                const bool in = q_in && t_in && a_in;
                const bool amb = q_amb || t_amb || a_amb;
                Hit h{t, alpha, e_t, e_alpha, base[k] + i, amb};
                if (in) hits.push_back(h);
                else if (amb) amb_out.push_back(h);
            }
        }
        std::sort(hits.begin(), hits.end(), [](const Hit& a, const Hit& b) { return a.t < b.t || (a.t == b.t && a.gid < b.gid); });
        // primary branch
        double T = 1.0, D = 0.0, sum_ea = 0.0;
        int comp = 0, amb = 0;
        size_t stop = hits.size();
        std::vector<double> Tin(hits.size(), 0.0), w(hits.size(), 0.0);
        double tA = 0.0, tD = 0.0;
        for (size_t i = 0; i < hits.size(); ++i) {
            const Hit& h = hits[i];
            const double Tn = T * (1.0 - h.alpha);
            sum_ea += h.alpha / (1.0 - h.alpha) * (h.e_alpha / std::max(h.alpha, 1e-300)) + 2 * kU;
            const double e_T = Tn * sum_ea + o->eps_rel * Tn;
            const bool term_amb = std::fabs(Tn - o->t_min) <= 2 * e_T;
            Tin[i] = T;
            if (term_amb) {
                double t_far = o->r_max;
                tA += T;
                tD += T * t_far;
                ++amb;
            }
            if (Tn < o->t_min) { stop = i; break; }
            w[i] = h.alpha * T;
            D += w[i] * h.t;
            T = Tn;
            ++comp;
        }
        const double A = 1.0 - T;
        // continuous errors
        for (size_t i = 0; i < stop; ++i) {
            tA += Tin[i] * hits[i].e_alpha;
            tD += w[i] * (hits[i].e_t + hits[i].t * hits[i].e_alpha / std::max(hits[i].alpha, 1e-300));
        }
        tD += 4 * kU * (double)comp * D;
        // ambiguous inclusions among the composited and among the left-out candidates
        auto behind = [&](double t) {     // primary D of the composited hits behind t
            double sum = 0.0;
            for (size_t i = 0; i < stop; ++i)
                if (hits[i].t > t) sum += w[i] * hits[i].t;
            return sum;
        };
        auto trans_at = [&](double t) {   // primary transmittance in front of t
            double Tt = 1.0;
            for (size_t i = 0; i < stop; ++i) {
                if (hits[i].t >= t) break;
                Tt *= 1.0 - hits[i].alpha;
            }
            return Tt;
        };
        for (size_t i = 0; i < hits.size(); ++i) {
            if (!hits[i].amb) continue;
            const double Tk = i < stop ? Tin[i] : trans_at(hits[i].t);
            tA += hits[i].alpha * Tk;
            tD += hits[i].alpha * (Tk * hits[i].t + behind(hits[i].t) / (1.0 - hits[i].alpha));
            ++amb;
        }
        for (const Hit& h : amb_out) {
            const double Tk = trans_at(h.t);
            tA += h.alpha * Tk;
            tD += h.alpha * (Tk * h.t + behind(h.t) / (1.0 - h.alpha));
            ++amb;
        }
        // near-ties in the order
        for (size_t i = 0; i + 1 < std::min(stop + 1, hits.size()); ++i) {
            const Hit &a = hits[i], &b = hits[i + 1];
            const double band = 2 * (a.e_t + b.e_t);
            if (b.t - a.t <= band) {
                const double wa = i < stop ? w[i] : 0.0, wb = i + 1 < stop ? w[i + 1] : 0.0;
                tD += (wa + wb + a.alpha * Tin[i]) * (b.t - a.t + band);
            }
        }
        out_d[ray] = D;
        out_a[ray] = A;
        tol_d[ray] = tD;
        tol_a[ray] = tA;
        n_comp[ray] = comp;
        n_amb[ray] = amb;
    });
    return 0;
}

}  // extern "C"
