// FP64 CPU oracle for batched 3D Gaussian Splatting RGB + depth rendering.
//
// TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or call this file:
// it exists so that tests/, the smoke check and the benchmark's CPU-baseline leg can check
// and time the CUDA renderer against an independent, slow, obviously correct definition.
// It shares no code, header or constant table with the CUDA library.
//
// What it computes (the plain definition the tile-binned GPU method must reproduce):
//   * Sec. III-B (Asset Formatting): every env holds a background node plus interactive
//     nodes; a node's Gaussians move rigidly with its world_from_node pose.
//   * Sec. III-A (Renderer): the native 3DGS pipeline -- per-Gaussian EWA splatting of the
//     3D covariance to a 2D conic, spherical-harmonics colour evaluation, depth ordering and
//     front-to-back alpha-blending.
//   * Sec. III-C (Sensor): RGB and depth are both produced by alpha-compositing, the colour
//     and the camera-space z of the intersected Gaussians respectively.
// For every pixel the oracle takes every Gaussian (of every node present in the env) whose
// centre is in front of the near plane and whose 3-sigma ellipse contains the pixel centre,
// sorts them by (depth, global id) and composites them front to back.  There is no tiling.
//
// Readings fixed where the paper is silent (every constant is an option in oracle_opts):
//   pixel centre (x+1/2, y+1/2); u = fx*tx/tz + cx; Sigma2D += lowpass*I; cull if tz <= z_near
//   or det(Sigma2D) <= 0; Jacobian evaluated at (tx/tz, ty/tz) clamped to +-guard*half-FOV
//   tangent; a Gaussian touches a pixel iff d^T conic d <= q_max (3 sigma -> 9);
//   alpha = min(alpha_max, opacity * exp(-q/2)); skip if alpha < alpha_min; T_next = T(1-alpha),
//   stop without compositing if T_next < t_min; RGB = sum w_i rgb_i + bg*T_final,
//   D = sum w_i z_i (unnormalised), A = 1 - T_final; real SH (Condon-Shortley phase) up to
//   degree 3, colour = max(0, sum c_lm Y_lm(d) + 1/2), d = unit view direction expressed in
//   the node frame.
//
// Depth order and the near-plane cull are decided on the FP64 camera-space z of the centre:
// candidates are sorted by (z, global id), global id = node_base[node] + local index, and culled
// when z <= z_near.  The method keeps its depth keys in FP32, so these two decisions are
// ambiguous where FP32 may take them the other way: the near cull when |z - z_near| lies within
// the error band of z, and the order of two candidates when their depths differ by less than the
// sum of their bands (an FP32 order may then place the later one first).  The method's FP32
// camera-space centre t (its z is the depth key) is taken to be rounded to binary32 within one
// unit in the last place per coordinate (faithful rounding, the accuracy of a compensated dot
// product; a key cannot be more accurate than the rounding of z itself), so the band of t_i is
// dt_i = 2u |t_i| + 64 u^2 S_i, u = 2^-24 (one ulp of t_i is at most 2u |t_i|; the second term,
// with S_i = sum_j |(Wc Rn)_ij mu_j| + |t_n| + |t_c,i| the magnitude of the summands, covers the
// residual error of the compensated sum with a factor 4 to spare).
//
// Every other decision is FP64 too.  A decision whose FP64 quantity lies within the FP32 error
// band of its threshold (ellipse, alpha_min, t_min) is likewise ambiguous.  The band is twice an
// error bound of the FP32 evaluation of that quantity: the projected centre carries
// dU ~ fx (d_tx + |x/z| d_tz)/z + 2u(|u| + |cx|) with d_t the band of t above;
// d_q = 2|dq/du| dU + 2|dq/dv| dV + 32u q (+ the error of the factored form); alpha moves by
// alpha (d_q/2 + (8 + 1.2|logit| + 0.6 q) u); the transmittance accumulates
// sum alpha/(1-alpha) d_alpha/alpha + 2u per step.  eps_rel adds a relative floor to every band.
// The forward pass enumerates up to max_flips flipped decisions per pixel along a branch (and at
// most max_branches branches per pixel) and returns every branch's result, each with the FP32
// error bound 2 T dT of its coverage A = 1 - T; beyond that it widens the pixel's tolerance by
// T * max|value| per unexplored flip (the two branches agree on the first 1-T of the composite
// and both stay inside the convex hull of the rest).  An order flip moves one later candidate,
// which may precede every acting candidate between, to the current position.

// The backward pass is the analytic adjoint of the primary branch (decisions held fixed).
// It is pinned by FP64 central finite differences of the forward pass in the tests.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <thread>
#include <vector>

extern "C" {

typedef struct {
    int32_t n_nodes;
    const int64_t* node_n;        // [n_nodes]
    const int32_t* node_deg;      // [n_nodes] SH degree 0..3
    const double* mean;           // [G,3]   G = sum(node_n), node-major
    const double* log_scale;      // [G,3]
    const double* quat;           // [G,4]   (w,x,y,z)
    const double* opacity_logit;  // [G]
    const double* sh;             // [G,16,3] (zero padded above the node's degree)
    int32_t E, K, C;
    const int32_t* env_node_ids;  // [E,K]   -1 = empty slot
    const double* node_poses;     // [E,K,12] world_from_node, row-major 3x4
    const int32_t* cams_per_env;  // [E]
    const double* cam_intr;       // [E,C,4] fx fy cx cy
    const int32_t* cam_res;       // [E,C,2] width height
    const double* cam_pose;       // [E,C,12] cam_from_world, row-major 3x4
} oracle_scene;

typedef struct {
    double z_near, lowpass, alpha_min, alpha_max, t_min, q_max, guard;
    double bg[3];
    double eps_rel;     // relative floor added to the FP32 error band of every decision
    int32_t max_flips;  // branches enumerated per pixel (<= 6)
    int32_t nthreads;   // 0 = hardware concurrency
    int32_t bruteforce; // 1 = test every Gaussian at every pixel (no AABB candidate lists)
    int32_t max_branches; // alternative branches enumerated per pixel before widening (0 = 64)
} oracle_opts;

}  // extern "C"

namespace {

constexpr double kPi = 3.14159265358979323846;

int n_threads(const oracle_opts* o) {
    if (o->nthreads > 0) return o->nthreads;
    unsigned h = std::thread::hardware_concurrency();
    return h ? (int)h : 1;
}

template <class F>
void parallel_for(int64_t n, int nth, F&& f) {
    if (n <= 0) return;
    std::atomic<int64_t> next(0);
    auto worker = [&](int tid) {
        for (;;) {
            int64_t i = next.fetch_add(1);
            if (i >= n) break;
            f(i, tid);
        }
    };
    nth = (int)std::max<int64_t>(1, std::min<int64_t>(nth, n));
    std::vector<std::thread> ts;
    for (int t = 1; t < nth; ++t) ts.emplace_back(worker, t);
    worker(0);
    for (auto& t : ts) t.join();
}

// ------------------------------------------------------------------ real spherical harmonics
// Sec. III-A (spherical-harmonics colour).  Y_lm for l <= 3 from the associated Legendre functions with the Condon-Shortley phase,
// written through Cartesian polynomials on the unit sphere:
//   P_l^m(cos t) e^{i m phi} = (-1)^m Q_l^m(z) (x + i y)^m,   Q_l^m = d^m P_l / dz^m,
//   Y_l0 = N_l0 Q_l^0,  Y_lm = sqrt2 N_lm (-1)^m Q_l^m Re[(x+iy)^m],
//   Y_l,-m = sqrt2 N_lm (-1)^m Q_l^m Im[(x+iy)^m],  N_lm = sqrt((2l+1)/(4 pi) (l-m)!/(l+m)!).
// Index k = l^2 + l + m.  The gradient is that of this polynomial extension to R^3; only its
// tangential part is used (after the normalisation Jacobian), which is unique.
double fact(int n) { double r = 1; for (int i = 2; i <= n; ++i) r *= i; return r; }

void sh_basis(int deg, const double d[3], double Y[16], double dY[16][3]) {
    const double x = d[0], y = d[1], z = d[2];
    double Q[5][5] = {{0}};   // Q[l][m] = m-th derivative of Legendre P_l at z (l<=3, m<=4)
    for (int m = 0; m <= 4; ++m) {
        for (int l = 0; l <= 3; ++l) {
            if (l < m) { Q[l][m] = 0; continue; }
            if (l == m) { double df = 1; for (int k = 2 * m - 1; k > 1; k -= 2) df *= k; Q[l][m] = df; continue; }
            if (l == m + 1) { Q[l][m] = (2 * m + 1) * z * Q[m][m]; continue; }
            Q[l][m] = ((2 * l - 1) * z * Q[l - 1][m] - (l + m - 1) * Q[l - 2][m]) / (l - m);
        }
    }
    double Cm[4], Sm[4];       // (x + i y)^m = Cm + i Sm
    Cm[0] = 1; Sm[0] = 0;
    for (int m = 1; m <= 3; ++m) { Cm[m] = Cm[m - 1] * x - Sm[m - 1] * y; Sm[m] = Cm[m - 1] * y + Sm[m - 1] * x; }
    for (int k = 0; k < 16; ++k) { Y[k] = 0; if (dY) dY[k][0] = dY[k][1] = dY[k][2] = 0; }
    for (int l = 0; l <= deg; ++l) {
        for (int m = -l; m <= l; ++m) {
            const int am = m < 0 ? -m : m;
            const int k = l * l + l + m;
            const double N = std::sqrt((2 * l + 1) / (4 * kPi) * fact(l - am) / fact(l + am));
            if (m == 0) {
                Y[k] = N * Q[l][0];
                if (dY) { dY[k][2] = N * Q[l][1]; }
                continue;
            }
            const double s = std::sqrt(2.0) * N * ((am & 1) ? -1.0 : 1.0);
            const double P = Q[l][am], dP = Q[l][am + 1];
            if (m > 0) {
                Y[k] = s * P * Cm[am];
                if (dY) { dY[k][0] = s * P * am * Cm[am - 1]; dY[k][1] = -s * P * am * Sm[am - 1]; dY[k][2] = s * dP * Cm[am]; }
            } else {
                Y[k] = s * P * Sm[am];
                if (dY) { dY[k][0] = s * P * am * Sm[am - 1]; dY[k][1] = s * P * am * Cm[am - 1]; dY[k][2] = s * dP * Sm[am]; }
            }
        }
    }
}

// ------------------------------------------------------------------ projection of one instance
struct Geo {
    int64_t gid;                 // global id = node_base + local
    int64_t g;                   // row in the concatenated attribute arrays (== gid)
    int slot, deg;
    double Rn[3][3], tn[3], mu[3], muw[3];
    double q[4], qlen, qn[4], Rq[3][3], sc[3], M[3][3], Sig[3][3], Sigw[3][3];
    double Wc[3][3], tc[3], t[3];
    double fx, fy, cx, cy, limx, limy, xr, yr, xc, yc;
    bool clx, cly;
    double J[2][3], T[2][3], cov[2][2], det, Q[2][2];
    double u, v, z, logit, opac;
    double dz;                   // FP32 error bound of z (order and near-plane decisions)
    double ocam[3], oloc[3], dir[3], dlen, d[3], Y[16], dY[16][3];
    double raw[3], rgb[3];
    bool present, near_amb, valid;
    double hx, hy;               // half extents of the ellipse's axis-aligned box (with band margin)
    double du, dv;               // FP32 error bound of the projected centre (pixels)
    bool grad_amb;               // a gradient switch (Jacobian guard, colour clamp) is within its FP32 band
    double dqb;                  // FP32 error bound of the factored form's cross coefficient
};

// Sec. III-A: the Gaussian's rotation from its quaternion (w, x, y, z), normalised first.
void rot_from_quat(const double q[4], double R[3][3]) {
    const double w = q[0], x = q[1], y = q[2], z = q[3];
    R[0][0] = 1 - 2 * (y * y + z * z); R[0][1] = 2 * (x * y - w * z); R[0][2] = 2 * (x * z + w * y);
    R[1][0] = 2 * (x * y + w * z); R[1][1] = 1 - 2 * (x * x + z * z); R[1][2] = 2 * (y * z - w * x);
    R[2][0] = 2 * (x * z - w * y); R[2][1] = 2 * (y * z + w * x); R[2][2] = 1 - 2 * (x * x + y * y);
}

// Sec. III-A (EWA splatting) with Sec. III-B's rigid node pose.  Projects Gaussian g (row in
// attribute arrays) of the node in `slot` of env e into camera (e, c).  Fills every intermediate.  valid=false if the 2D covariance is not positive.
void project(const oracle_scene* s, const oracle_opts* o, int e, int c, int slot, int64_t g, int deg, Geo& G) {
    G.g = g; G.gid = g; G.slot = slot; G.deg = deg;
    const double* P = s->node_poses + ((int64_t)e * s->K + slot) * 12;
    for (int i = 0; i < 3; ++i) { for (int j = 0; j < 3; ++j) G.Rn[i][j] = P[i * 4 + j]; G.tn[i] = P[i * 4 + 3]; }
    const double* CP = s->cam_pose + ((int64_t)e * s->C + c) * 12;
    for (int i = 0; i < 3; ++i) { for (int j = 0; j < 3; ++j) G.Wc[i][j] = CP[i * 4 + j]; G.tc[i] = CP[i * 4 + 3]; }
    const double* I = s->cam_intr + ((int64_t)e * s->C + c) * 4;
    G.fx = I[0]; G.fy = I[1]; G.cx = I[2]; G.cy = I[3];
    const int32_t* res = s->cam_res + ((int64_t)e * s->C + c) * 2;
    G.limx = o->guard * 0.5 * res[0] / G.fx;
    G.limy = o->guard * 0.5 * res[1] / G.fy;

    for (int i = 0; i < 3; ++i) G.mu[i] = s->mean[g * 3 + i];
    for (int i = 0; i < 3; ++i) G.muw[i] = G.Rn[i][0] * G.mu[0] + G.Rn[i][1] * G.mu[1] + G.Rn[i][2] * G.mu[2] + G.tn[i];
    // 3D covariance in the node frame: Sigma = R(q) S S^T R(q)^T, S = diag(exp(log_scale)).
    for (int i = 0; i < 4; ++i) G.q[i] = s->quat[g * 4 + i];
    G.qlen = std::sqrt(G.q[0] * G.q[0] + G.q[1] * G.q[1] + G.q[2] * G.q[2] + G.q[3] * G.q[3]);
    for (int i = 0; i < 4; ++i) G.qn[i] = G.q[i] / G.qlen;
    rot_from_quat(G.qn, G.Rq);
    for (int i = 0; i < 3; ++i) G.sc[i] = std::exp(s->log_scale[g * 3 + i]);
    for (int i = 0; i < 3; ++i) for (int j = 0; j < 3; ++j) G.M[i][j] = G.Rq[i][j] * G.sc[j];
    for (int i = 0; i < 3; ++i) for (int j = 0; j < 3; ++j) {
        double a = 0; for (int k = 0; k < 3; ++k) a += G.M[i][k] * G.M[j][k]; G.Sig[i][j] = a; }
    // World covariance Sigma_w = Rn Sigma Rn^T.
    double tmp[3][3];
    for (int i = 0; i < 3; ++i) for (int j = 0; j < 3; ++j) {
        double a = 0; for (int k = 0; k < 3; ++k) a += G.Rn[i][k] * G.Sig[k][j]; tmp[i][j] = a; }
    for (int i = 0; i < 3; ++i) for (int j = 0; j < 3; ++j) {
        double a = 0; for (int k = 0; k < 3; ++k) a += tmp[i][k] * G.Rn[j][k]; G.Sigw[i][j] = a; }
    // Camera space.
    for (int i = 0; i < 3; ++i) G.t[i] = G.Wc[i][0] * G.muw[0] + G.Wc[i][1] * G.muw[1] + G.Wc[i][2] * G.muw[2] + G.tc[i];
    G.z = G.t[2];
    const double g32 = 5.9604644775390625e-08;
    double MR[3][3];
    for (int i = 0; i < 3; ++i) for (int j = 0; j < 3; ++j) {
        double a = 0; for (int k = 0; k < 3; ++k) a += G.Wc[i][k] * G.Rn[k][j]; MR[i][j] = a; }
    const double tnn = std::sqrt(G.tn[0] * G.tn[0] + G.tn[1] * G.tn[1] + G.tn[2] * G.tn[2]);
    double S[3];   // magnitude of the terms summed into each camera-space coordinate
    for (int i = 0; i < 3; ++i)
        S[i] = std::fabs(MR[i][0] * G.mu[0]) + std::fabs(MR[i][1] * G.mu[1]) + std::fabs(MR[i][2] * G.mu[2]) +
               tnn + std::fabs(G.tc[i]);
    double dt[3];   // FP32 error bounds of the camera-space centre (faithful rounding, twice)
    for (int i = 0; i < 3; ++i) dt[i] = 2 * g32 * std::fabs(G.t[i]) + 64 * g32 * g32 * S[i];
    G.dz = dt[2];
    // near plane: FP64 decision, ambiguous within the band of z (and the FP32 rounding of z_near)
    G.present = G.z > o->z_near;
    G.near_amb = std::fabs(G.z - o->z_near) <= G.dz + 2 * g32 * o->z_near + o->eps_rel * o->z_near;
    G.valid = true;
    G.grad_amb = false;
    if (!G.present && !G.near_amb) { G.valid = false; return; }
    // EWA: Jacobian of the pinhole projection at t (guarded), Sigma2D = J Wc Sigma_w Wc^T J^T + lp I.
    G.xr = G.t[0] / G.t[2]; G.yr = G.t[1] / G.t[2];
    G.xc = std::min(G.limx, std::max(-G.limx, G.xr)); G.clx = G.xc != G.xr;
    G.yc = std::min(G.limy, std::max(-G.limy, G.yr)); G.cly = G.yc != G.yr;
    G.J[0][0] = G.fx / G.t[2]; G.J[0][1] = 0; G.J[0][2] = -G.fx * G.xc / G.t[2];
    G.J[1][0] = 0; G.J[1][1] = G.fy / G.t[2]; G.J[1][2] = -G.fy * G.yc / G.t[2];
    for (int i = 0; i < 2; ++i) for (int j = 0; j < 3; ++j) {
        double a = 0; for (int k = 0; k < 3; ++k) a += G.J[i][k] * G.Wc[k][j]; G.T[i][j] = a; }
    double TS[2][3];
    for (int i = 0; i < 2; ++i) for (int j = 0; j < 3; ++j) {
        double a = 0; for (int k = 0; k < 3; ++k) a += G.T[i][k] * G.Sigw[k][j]; TS[i][j] = a; }
    for (int i = 0; i < 2; ++i) for (int j = 0; j < 2; ++j) {
        double a = 0; for (int k = 0; k < 3; ++k) a += TS[i][k] * G.T[j][k]; G.cov[i][j] = a; }
    G.cov[0][0] += o->lowpass; G.cov[1][1] += o->lowpass;
    G.det = G.cov[0][0] * G.cov[1][1] - G.cov[0][1] * G.cov[1][0];
    if (!(G.det > 0)) { G.valid = false; return; }
    G.Q[0][0] = G.cov[1][1] / G.det; G.Q[1][1] = G.cov[0][0] / G.det;
    G.Q[0][1] = G.Q[1][0] = -G.cov[0][1] / G.det;
    G.u = G.fx * G.xr + G.cx; G.v = G.fy * G.yr + G.cy;
    {   // FP32 error model of the projected centre
        const double dtx = dt[0], dty = dt[1], dtz = dt[2];
        const double dxr = (dtx + std::fabs(G.xr) * dtz) / G.t[2] + 2 * g32 * std::fabs(G.xr);
        const double dyr = (dty + std::fabs(G.yr) * dtz) / G.t[2] + 2 * g32 * std::fabs(G.yr);
        G.du = G.fx * dxr + 2 * g32 * (std::fabs(G.fx * G.xr) + std::fabs(G.cx));
        G.dv = G.fy * dyr + 2 * g32 * (std::fabs(G.fy * G.yr) + std::fabs(G.cy));
        // the guard clamps xr at +-limx: its gradient switches there
        G.grad_amb = std::fabs(std::fabs(G.xr) - G.limx) <= 2 * dxr + 4 * g32 * G.limx ||
                     std::fabs(std::fabs(G.yr) - G.limy) <= 2 * dyr + 4 * g32 * G.limy;
        G.dqb = 8 * g32 * std::sqrt(G.cov[0][0] / G.cov[1][1]);
    }
    // Bounding box of {d : d^T Q d <= qb}, a superset of every candidate whose band reaches q_max.
    const double qb = o->q_max * (1.01 + 2.0 * o->eps_rel) + 0.1;
    G.hx = std::sqrt(qb * G.cov[0][0]) * (1 + 1e-12) + 1e-12;
    G.hy = std::sqrt(qb * G.cov[1][1]) * (1 + 1e-12) + 1e-12;
    // Opacity.
    G.logit = s->opacity_logit[g];
    G.opac = 1.0 / (1.0 + std::exp(-G.logit));
    // View direction in the node frame: camera centre o = -Wc^T tc, o_local = Rn^T (o - tn).
    for (int i = 0; i < 3; ++i) G.ocam[i] = -(G.Wc[0][i] * G.tc[0] + G.Wc[1][i] * G.tc[1] + G.Wc[2][i] * G.tc[2]);
    for (int i = 0; i < 3; ++i) {
        double a = 0; for (int k = 0; k < 3; ++k) a += G.Rn[k][i] * (G.ocam[k] - G.tn[k]); G.oloc[i] = a; }
    for (int i = 0; i < 3; ++i) G.dir[i] = G.mu[i] - G.oloc[i];
    G.dlen = std::sqrt(G.dir[0] * G.dir[0] + G.dir[1] * G.dir[1] + G.dir[2] * G.dir[2]);
    for (int i = 0; i < 3; ++i) G.d[i] = G.dir[i] / G.dlen;
    sh_basis(deg, G.d, G.Y, G.dY);
    const double* sh = s->sh + g * 48;
    for (int ch = 0; ch < 3; ++ch) {
        double a = 0.5, mag = 0.5;
        for (int k = 0; k < (deg + 1) * (deg + 1); ++k) { a += sh[k * 3 + ch] * G.Y[k]; mag += std::fabs(sh[k * 3 + ch] * G.Y[k]); }
        G.raw[ch] = a; G.rgb[ch] = a > 0 ? a : 0.0;
        // the colour clamp at 0 switches the colour gradient: FP32 band of the sum
        if (std::fabs(a) <= 64 * 5.9604644775390625e-08 * mag) G.grad_amb = true;
    }
}

struct ViewData {
    int W = 0, H = 0;
    std::vector<Geo> geo;        // instances that are present or near-ambiguous and valid
    std::vector<int64_t> node_base;
};

bool build_view(const oracle_scene* s, const oracle_opts* o, int e, int c, ViewData& V) {
    if (e < 0 || e >= s->E || c < 0 || c >= s->cams_per_env[e]) return false;
    const int32_t* res = s->cam_res + ((int64_t)e * s->C + c) * 2;
    V.W = res[0]; V.H = res[1];
    V.node_base.assign(s->n_nodes + 1, 0);
    for (int k = 0; k < s->n_nodes; ++k) V.node_base[k + 1] = V.node_base[k] + s->node_n[k];
    // Instances in slot order; the id used for ordering is the global id.
    std::vector<std::pair<int, int64_t>> items;   // (slot, g)
    for (int j = 0; j < s->K; ++j) {
        int k = s->env_node_ids[(int64_t)e * s->K + j];
        if (k < 0) continue;
        for (int64_t i = 0; i < s->node_n[k]; ++i) items.emplace_back(j, V.node_base[k] + i);
    }
    std::vector<Geo> all(items.size());
    std::vector<char> keep(items.size(), 0);
    parallel_for((int64_t)items.size(), n_threads(o), [&](int64_t i, int) {
        const int slot = items[i].first;
        const int k = s->env_node_ids[(int64_t)e * s->K + slot];
        project(s, o, e, c, slot, items[i].second, s->node_deg[k], all[i]);
        keep[i] = all[i].valid;
    });
    V.geo.clear();
    for (size_t i = 0; i < all.size(); ++i) if (keep[i]) V.geo.push_back(all[i]);
    return true;
}

// Per-pixel candidate: a Gaussian whose band-widened ellipse contains the pixel centre, with the
// decisions that do not depend on the transmittance: near plane, ellipse and alpha_min (d) and
// whether FP32 may take each the other way (amb).
struct Cand {
    int idx;
    double z, dz;                 // FP64 depth and its FP32 error bound
    int64_t gid;
    double q, dx, dy, dq;         // quadratic form at the pixel and its FP32 error bound
    double a_raw, alpha, da;      // opacity * exp(-q/2), its clamp, relative FP32 error bound
    bool d[3], amb[3];
    bool may_act;                 // composited or stopping under some admissible decision
};

void pixel_candidates(const ViewData& V, const oracle_opts* o, const std::vector<int>& pool, int px, int py,
                      std::vector<Cand>& out) {
    out.clear();
    const double X = px + 0.5, Yc = py + 0.5;
    const double qlim = o->q_max * (1.01 + 2.0 * o->eps_rel) + 0.1;
    const double g32 = 5.9604644775390625e-08;
    const double eps = o->eps_rel;
    for (int idx : pool) {
        const Geo& G = V.geo[idx];
        const double dx = X - G.u, dy = Yc - G.v;
        const double q = G.Q[0][0] * dx * dx + 2 * G.Q[0][1] * dx * dy + G.Q[1][1] * dy * dy;
        if (q > qlim) continue;
        // FP32 error bound of q at this pixel: centre error, factored-form coefficient, rounding
        const double t = dx - (G.cov[0][1] / G.cov[1][1]) * dy;
        const double dq = 2 * (std::fabs(G.Q[0][0] * dx + G.Q[0][1] * dy) * G.du + std::fabs(G.Q[0][1] * dx + G.Q[1][1] * dy) * G.dv) +
                          2 * G.Q[0][0] * std::fabs(t * dy) * G.dqb + 32 * g32 * q + 1e-9;
        Cand c;
        c.idx = idx; c.z = G.z; c.dz = G.dz; c.gid = G.gid; c.q = q; c.dx = dx; c.dy = dy; c.dq = dq;
        c.a_raw = G.opac * std::exp(-0.5 * q);
        c.alpha = std::min(o->alpha_max, c.a_raw);
        c.da = (c.a_raw > o->alpha_max) ? 4 * g32 : 0.5 * dq + (8 + 1.2 * std::fabs(G.logit) + 0.6 * q) * g32;
        c.d[0] = G.present; c.d[1] = q <= o->q_max; c.d[2] = c.alpha >= o->alpha_min;
        c.amb[0] = G.near_amb;
        c.amb[1] = std::fabs(q - o->q_max) <= 2 * dq + eps * o->q_max;
        c.amb[2] = std::fabs(c.alpha - o->alpha_min) <= 2 * c.alpha * c.da + eps * o->alpha_min;
        c.may_act = (c.d[0] || c.amb[0]) && (c.d[1] || c.amb[1]) && (c.d[2] || c.amb[2]);
        out.push_back(c);
    }
    std::sort(out.begin(), out.end(), [](const Cand& a, const Cand& b) {
        return a.z < b.z || (a.z == b.z && a.gid < b.gid); });
}

// May an FP32 evaluation of the two depths place candidate b (after a in FP64 order) first?
inline bool may_precede(const Cand& a, const Cand& b, double eps) {
    return b.z - a.z <= a.dz + b.dz + eps * std::fabs(a.z);
}

// One composite: colour, depth, coverage and the FP32 error bound 2 T dT of the coverage.
struct Leaf { double r, g, b, d, a, ea; };

struct PixelResult {
    Leaf primary;
    std::vector<Leaf> alts;
    double tol_rgb = 0, tol_d = 0;
    bool ambiguous = false;
    bool widened = false;                 // a flip beyond the branch budget widened the tolerance
    int64_t amb_kind[5] = {0, 0, 0, 0, 0};   // near, ellipse, alpha, transmittance, depth order
    bool grad_amb = false;                // a gradient switch of a contributor lies within its FP32 band
    int64_t contrib = 0;                  // Gaussians composited (primary branch)
    int64_t reached = 0;                  // in-ellipse Gaussians reached before termination (primary)
    bool terminated = false;
    uint64_t hash = 1469598103934665603ull;
};

inline uint64_t mix(uint64_t h, uint64_t v) { h ^= v + 0x9e3779b97f4a7c15ull + (h << 6) + (h >> 2); return h * 1099511628211ull; }

// Sec. III-A (alpha-blending) and Sec. III-C (depth from the composited z).  Front-to-back
// composite of one pixel, branching on ambiguous decisions.
// A candidate's action is SKIP unless it is in front of the near plane, inside the ellipse and
// has alpha >= alpha_min; then it is STOP if T(1-alpha) < t_min, else COMPOSITE.  Flipping one
// ambiguous decision that changes the action starts an alternative branch; so does placing a
// later candidate first whose depth ties with every acting candidate before it (the order
// decision).
enum Act { SKIP = 0, COMP = 1, STOP = 2 };

inline Act action(bool near_ok, bool ell_ok, bool keep, bool stop) {
    if (!(near_ok && ell_ok && keep)) return SKIP;
    return stop ? STOP : COMP;
}

struct Compositor {
    const ViewData& V; const oracle_opts* o;
    double Mc, Mz, dz_max;
    size_t max_branches;
    PixelResult* R;

    void widen(double T) { R->tol_rgb += T * Mc; R->tol_d += T * Mz; R->widened = true; }
    bool budget(int flips) const { return flips < o->max_flips && R->alts.size() < max_branches; }

    // fixed: the candidate at `pos` was placed there by an order flip of this branch (its order
    // decision is taken)
    void run(const std::vector<Cand>& order, size_t pos, double T, double C0, double C1, double C2, double D,
             int flips, bool primary, double dT, bool fixed) {
        const double eps = o->eps_rel;
        const double g32 = 5.9604644775390625e-08;
        for (; pos < order.size(); ++pos, fixed = false) {
            const Cand& cd = order[pos];
            const Geo& G = V.geo[cd.idx];
            if (!fixed && cd.may_act) {
                // order decisions: a later candidate that may act and may precede every acting
                // candidate from here to it
                for (size_t j = pos + 1; j < order.size(); ++j) {
                    const Cand& cj = order[j];
                    if (cj.z - cd.z > cd.dz + dz_max + eps * std::fabs(cd.z)) break;
                    if (!cj.may_act) continue;
                    bool tie = true;
                    for (size_t i = pos; i < j && tie; ++i) tie = !order[i].may_act || may_precede(order[i], cj, eps);
                    if (!tie) continue;
                    R->ambiguous = true;
                    if (primary) R->amb_kind[4]++;
                    if (!budget(flips)) { widen(T); continue; }
                    std::vector<Cand> alt(order);
                    std::rotate(alt.begin() + pos, alt.begin() + j, alt.begin() + j + 1);
                    run(alt, pos, T, C0, C1, C2, D, flips + 1, false, dT, true);
                }
            }
            const double alpha = cd.alpha;
            const double Tn = T * (1.0 - alpha);
            // relative FP32 error bound of T after this Gaussian
            const double dTn = dT + alpha / (1.0 - alpha) * cd.da + 2 * g32;
            const bool d[4] = {cd.d[0], cd.d[1], cd.d[2], Tn < o->t_min};
            const bool amb[4] = {cd.amb[0], cd.amb[1], cd.amb[2], std::fabs(Tn - o->t_min) <= 2 * Tn * dTn + eps * o->t_min};
            const Act act = action(d[0], d[1], d[2], d[3]);
            for (int k = 0; k < 4; ++k) {
                if (!amb[k]) continue;
                bool f[4] = {d[0], d[1], d[2], d[3]};
                f[k] = !f[k];
                const Act alt = action(f[0], f[1], f[2], f[3]);
                if (alt == act) continue;
                R->ambiguous = true;
                if (primary) R->amb_kind[k]++;
                if (!budget(flips)) { widen(T); continue; }
                if (alt == SKIP) run(order, pos + 1, T, C0, C1, C2, D, flips + 1, false, dT, false);
                else if (alt == STOP) emit(T, C0, C1, C2, D, dT, false);
                else {
                    const double w = alpha * T;
                    run(order, pos + 1, Tn, C0 + w * G.rgb[0], C1 + w * G.rgb[1], C2 + w * G.rgb[2], D + w * G.z,
                        flips + 1, false, dTn, false);
                }
            }
            if (primary) {
                uint64_t code = (uint64_t)act;
                if (act != SKIP) code += 4 * (cd.a_raw > o->alpha_max) + 8 * (G.clx || G.cly) + 16 * (G.raw[0] <= 0) +
                                         32 * (G.raw[1] <= 0) + 64 * (G.raw[2] <= 0);
                R->hash = mix(R->hash, (uint64_t)cd.gid * 128 + code);
            }
            if (primary && d[0] && d[1]) R->reached++;
            if (act == SKIP) continue;
            if (act == STOP) { if (primary) R->terminated = true; break; }
            if (primary) {
                R->contrib++;
                // alpha clamp at alpha_max: continuous value, switched gradient
                if (G.grad_amb || std::fabs(cd.a_raw - o->alpha_max) <= 2 * cd.a_raw * cd.da + eps * o->alpha_max)
                    R->grad_amb = true;
            }
            const double w = alpha * T;
            C0 += w * G.rgb[0]; C1 += w * G.rgb[1]; C2 += w * G.rgb[2]; D += w * G.z;
            T = Tn;
            dT = dTn;
        }
        emit(T, C0, C1, C2, D, dT, primary);
    }
    void emit(double T, double C0, double C1, double C2, double D, double dT, bool primary) {
        Leaf L{C0 + o->bg[0] * T, C1 + o->bg[1] * T, C2 + o->bg[2] * T, D, 1.0 - T, 2 * T * dT};
        if (primary) R->primary = L; else R->alts.push_back(L);
    }
};

// Row buckets: for every pixel row, the instances whose box covers a pixel centre of that row.
void row_pools(const ViewData& V, const oracle_opts* o, std::vector<std::vector<int>>& rows) {
    rows.assign(V.H, {});
    for (int i = 0; i < (int)V.geo.size(); ++i) {
        const Geo& G = V.geo[i];
        if (o->bruteforce) { for (int y = 0; y < V.H; ++y) rows[y].push_back(i); continue; }
        // rows y with |y + 0.5 - v| <= hy
        double lo = std::ceil(G.v - G.hy - 0.5), hi = std::floor(G.v + G.hy - 0.5);
        if (hi < 0 || lo > V.H - 1) continue;
        int y0 = (int)std::max(0.0, lo), y1 = (int)std::min((double)V.H - 1, hi);
        for (int y = y0; y <= y1; ++y) rows[y].push_back(i);
    }
}

void cols_pool(const ViewData& V, const oracle_opts* o, const std::vector<int>& row, std::vector<std::vector<int>>& cols) {
    for (auto& c : cols) c.clear();
    for (int i : row) {
        const Geo& G = V.geo[i];
        if (o->bruteforce) { for (int x = 0; x < V.W; ++x) cols[x].push_back(i); continue; }
        double lo = std::ceil(G.u - G.hx - 0.5), hi = std::floor(G.u + G.hx - 0.5);
        if (hi < 0 || lo > V.W - 1) continue;
        int x0 = (int)std::max(0.0, lo), x1 = (int)std::min((double)V.W - 1, hi);
        for (int x = x0; x <= x1; ++x) cols[x].push_back(i);
    }
}

// Sec. IV: attribute and pose gradients of one instance from its 10 per-instance partials r
// (u, v, conic a, b, c, opacity, r, g, b, z): the chain rule through projection, colour and pose.
struct InstGrad {
    double mean[3] = {0, 0, 0}, log_scale[3] = {0, 0, 0}, quat[4] = {0, 0, 0, 0}, logit = 0, sh[48] = {0}, pose[12] = {0};
};

void chain_rule(const oracle_scene* s, const Geo& G, const double r[10], InstGrad& out) {
    const int64_t g = G.g;
    double gRn[3][3] = {{0}}, gtn[3] = {0}, gmu[3] = {0};
    // opacity
    out.logit += r[5] * G.opac * (1 - G.opac);
    // colour: rgb = max(0, sum c_k Y_k(d) + 1/2)
    double gd[3] = {0, 0, 0};
    const int nc = (G.deg + 1) * (G.deg + 1);
    for (int ch = 0; ch < 3; ++ch) {
        if (!(G.raw[ch] > 0)) continue;
        const double gr = r[6 + ch];
        for (int k = 0; k < nc; ++k) {
            out.sh[k * 3 + ch] += gr * G.Y[k];
            const double cf = s->sh[g * 48 + k * 3 + ch];
            for (int j = 0; j < 3; ++j) gd[j] += gr * cf * G.dY[k][j];
        }
    }
    const double dd = gd[0] * G.d[0] + gd[1] * G.d[1] + gd[2] * G.d[2];
    double gdir[3];
    for (int j = 0; j < 3; ++j) gdir[j] = (gd[j] - G.d[j] * dd) / G.dlen;
    for (int j = 0; j < 3; ++j) gmu[j] += gdir[j];
    // dir = mu - o_local, o_local = Rn^T (o - tn)
    for (int a = 0; a < 3; ++a) for (int b = 0; b < 3; ++b) gRn[a][b] += (G.ocam[a] - G.tn[a]) * (-gdir[b]);
    for (int a = 0; a < 3; ++a) { double v = 0; for (int b = 0; b < 3; ++b) v += G.Rn[a][b] * (-gdir[b]); gtn[a] -= v; }
    // conic -> 2D covariance: gCov = -Q G Q with G = [[ga, gb/2],[gb/2, gc]]
    const double Gm[2][2] = {{r[2], 0.5 * r[3]}, {0.5 * r[3], r[4]}};
    double QG[2][2], gCov[2][2];
    for (int a = 0; a < 2; ++a) for (int b = 0; b < 2; ++b) QG[a][b] = G.Q[a][0] * Gm[0][b] + G.Q[a][1] * Gm[1][b];
    for (int a = 0; a < 2; ++a) for (int b = 0; b < 2; ++b) gCov[a][b] = -(QG[a][0] * G.Q[0][b] + QG[a][1] * G.Q[1][b]);
    // Cov = T Sigma_w T^T + lp I:  gSigma_w = T^T gCov T,  gT = 2 gCov T Sigma_w
    double gSigw[3][3], gT[2][3];
    for (int a = 0; a < 3; ++a) for (int b = 0; b < 3; ++b) {
        double v = 0; for (int m = 0; m < 2; ++m) for (int n = 0; n < 2; ++n) v += G.T[m][a] * gCov[m][n] * G.T[n][b];
        gSigw[a][b] = v; }
    for (int a = 0; a < 2; ++a) for (int b = 0; b < 3; ++b) {
        double v = 0;
        for (int m = 0; m < 2; ++m) for (int k = 0; k < 3; ++k) v += gCov[a][m] * G.T[m][k] * G.Sigw[k][b];
        gT[a][b] = 2 * v; }
    // T = J Wc: gJ = gT Wc^T
    double gJ[2][3];
    for (int a = 0; a < 2; ++a) for (int b = 0; b < 3; ++b) {
        double v = 0; for (int k = 0; k < 3; ++k) v += gT[a][k] * G.Wc[b][k]; gJ[a][b] = v; }
    double gt[3] = {0, 0, 0};
    const double tx = G.t[0], ty = G.t[1], tz = G.t[2];
    gt[2] += gJ[0][0] * (-G.fx / (tz * tz)) + gJ[1][1] * (-G.fy / (tz * tz));
    if (!G.clx) { gt[2] += gJ[0][2] * (2 * G.fx * tx / (tz * tz * tz)); gt[0] += gJ[0][2] * (-G.fx / (tz * tz)); }
    else { gt[2] += gJ[0][2] * (G.fx * G.xc / (tz * tz)); }
    if (!G.cly) { gt[2] += gJ[1][2] * (2 * G.fy * ty / (tz * tz * tz)); gt[1] += gJ[1][2] * (-G.fy / (tz * tz)); }
    else { gt[2] += gJ[1][2] * (G.fy * G.yc / (tz * tz)); }
    // mean in pixels and depth
    gt[0] += r[0] * G.fx / tz; gt[2] += -r[0] * G.fx * tx / (tz * tz);
    gt[1] += r[1] * G.fy / tz; gt[2] += -r[1] * G.fy * ty / (tz * tz);
    gt[2] += r[9];
    // t = Wc mu_w + tc; mu_w = Rn mu + tn
    double gmuw[3];
    for (int a = 0; a < 3; ++a) gmuw[a] = G.Wc[0][a] * gt[0] + G.Wc[1][a] * gt[1] + G.Wc[2][a] * gt[2];
    for (int a = 0; a < 3; ++a) { gtn[a] += gmuw[a]; for (int b = 0; b < 3; ++b) { gRn[a][b] += gmuw[a] * G.mu[b]; gmu[b] += G.Rn[a][b] * gmuw[a]; } }
    // Sigma_w = Rn Sigma Rn^T: gSigma = Rn^T gSigw Rn, gRn += 2 gSigw Rn Sigma
    double gSig[3][3], tmp[3][3];
    for (int a = 0; a < 3; ++a) for (int b = 0; b < 3; ++b) { double v = 0; for (int k = 0; k < 3; ++k) v += gSigw[a][k] * G.Rn[k][b]; tmp[a][b] = v; }
    for (int a = 0; a < 3; ++a) for (int b = 0; b < 3; ++b) { double v = 0; for (int k = 0; k < 3; ++k) v += G.Rn[k][a] * tmp[k][b]; gSig[a][b] = v; }
    for (int a = 0; a < 3; ++a) for (int b = 0; b < 3; ++b) { double v = 0; for (int k = 0; k < 3; ++k) v += tmp[a][k] * G.Sig[k][b]; gRn[a][b] += 2 * v; }
    // Sigma = M M^T, M = Rq diag(sc): gM = 2 gSigma M
    double gM[3][3];
    for (int a = 0; a < 3; ++a) for (int b = 0; b < 3; ++b) { double v = 0; for (int k = 0; k < 3; ++k) v += gSig[a][k] * G.M[k][b]; gM[a][b] = 2 * v; }
    for (int j = 0; j < 3; ++j) { double v = 0; for (int i2 = 0; i2 < 3; ++i2) v += G.Rq[i2][j] * gM[i2][j]; out.log_scale[j] += v * G.sc[j]; }
    double gRq[3][3];
    for (int a = 0; a < 3; ++a) for (int b = 0; b < 3; ++b) gRq[a][b] = gM[a][b] * G.sc[b];
    // Rq(qn) -> qn
    const double w = G.qn[0], x = G.qn[1], yq = G.qn[2], zq = G.qn[3];
    const double dRw[3][3] = {{0, -2 * zq, 2 * yq}, {2 * zq, 0, -2 * x}, {-2 * yq, 2 * x, 0}};
    const double dRx[3][3] = {{0, 2 * yq, 2 * zq}, {2 * yq, -4 * x, -2 * w}, {2 * zq, 2 * w, -4 * x}};
    const double dRy[3][3] = {{-4 * yq, 2 * x, 2 * w}, {2 * x, 0, 2 * zq}, {-2 * w, 2 * zq, -4 * yq}};
    const double dRz[3][3] = {{-4 * zq, -2 * w, 2 * x}, {2 * w, -4 * zq, 2 * yq}, {2 * x, 2 * yq, 0}};
    double gqn[4] = {0, 0, 0, 0};
    for (int a = 0; a < 3; ++a) for (int b = 0; b < 3; ++b) {
        gqn[0] += gRq[a][b] * dRw[a][b]; gqn[1] += gRq[a][b] * dRx[a][b];
        gqn[2] += gRq[a][b] * dRy[a][b]; gqn[3] += gRq[a][b] * dRz[a][b]; }
    const double qd = gqn[0] * G.qn[0] + gqn[1] * G.qn[1] + gqn[2] * G.qn[2] + gqn[3] * G.qn[3];
    for (int k = 0; k < 4; ++k) out.quat[k] += (gqn[k] - G.qn[k] * qd) / G.qlen;
    for (int k = 0; k < 3; ++k) out.mean[k] += gmu[k];
    for (int a = 0; a < 3; ++a) { for (int b = 0; b < 3; ++b) out.pose[a * 4 + b] += gRn[a][b]; out.pose[a * 4 + 3] += gtn[a]; }
}

}  // namespace

extern "C" {

int oracle_abi_version() { return 1; }

// Sec. III-A: real SH basis Y[16] (entries above the degree are 0) and its gradient dY[16][3] at d.
void oracle_sh_basis(int deg, const double* d, double* Y, double* dY) {
    double y[16], dy[16][3];
    sh_basis(deg, d, y, dy);
    for (int k = 0; k < 16; ++k) { Y[k] = y[k]; if (dY) for (int j = 0; j < 3; ++j) dY[k * 3 + j] = dy[k][j]; }
}

// Sec. III-A: projection of every Gaussian of view (e, c), for closed-form checks.
// out[n, 16]: gid, u, v, z, conic a, b, c, cov xx, xy, yy, opacity, r, g, b, present, near_amb.
// Returns the number of valid instances written (<= cap), or -1 on bad arguments.
int64_t oracle_project_view(const oracle_scene* s, const oracle_opts* o, int e, int c, double* out, int64_t cap) {
    ViewData V;
    if (!build_view(s, o, e, c, V)) return -1;
    int64_t n = 0;
    for (const Geo& G : V.geo) {
        if (n >= cap) break;
        double* r = out + n * 16;
        r[0] = (double)G.gid; r[1] = G.u; r[2] = G.v; r[3] = G.z;
        r[4] = G.Q[0][0]; r[5] = G.Q[0][1]; r[6] = G.Q[1][1];
        r[7] = G.cov[0][0]; r[8] = G.cov[0][1]; r[9] = G.cov[1][1];
        r[10] = G.opac; r[11] = G.rgb[0]; r[12] = G.rgb[1]; r[13] = G.rgb[2];
        r[14] = G.present; r[15] = G.near_amb;
        ++n;
    }
    return (int64_t)V.geo.size();
}

// Sec. III-A and III-C: renders view (e, c).  rgb [H*W*3], depth/alpha [H*W]: the primary branch.
// err_a [H*W] (nullable): FP32 error bound of the primary branch's coverage.
// tol_rgb/tol_d [H*W]: extra tolerance from flips beyond the branch budget.  n_alt [H*W]: number
// of alternative branches of each pixel; alt [alt_cap*6] receives them (r, g, b, d, a, error
// bound of a) in pixel order.  grad_amb [H*W] (nullable) marks pixels where a contributor's
// gradient switch (alpha clamp, Jacobian guard, colour clamp) lies within its FP32 band.
// stats[0] = alternatives needed, stats[1] = ambiguous pixels, stats[2] = decision hash (as
// bits), stats[3] = instances projected, stats[4..7] = ambiguous decisions on the primary branch
// by kind (near plane, ellipse, alpha_min, t_min), stats[8] = Gaussians composited, stats[9] =
// in-ellipse Gaussians reached before termination, stats[10] = pixels that terminated (all on
// the primary branch), stats[11] = ambiguous depth-order decisions on the primary branch,
// stats[12] = pixels whose tolerance was widened; stats needs 13 entries.  Returns 0, or -1 on
// bad arguments, or 1 if alt_cap was too small (outputs other than alt are still complete).
int oracle_render_view(const oracle_scene* s, const oracle_opts* o, int e, int c,
                       double* rgb, double* depth, double* alpha, double* err_a, double* tol_rgb, double* tol_d,
                       int32_t* n_alt, double* alt, int64_t alt_cap, int64_t* stats, int32_t* grad_amb) {
    ViewData V;
    if (!build_view(s, o, e, c, V)) return -1;
    std::vector<std::vector<int>> rows;
    row_pools(V, o, rows);
    const int W = V.W, H = V.H;
    const size_t max_branches = o->max_branches > 0 ? (size_t)o->max_branches : 64;
    std::vector<std::vector<Leaf>> row_alts(H);
    std::vector<int64_t> row_amb(H, 0), row_wide(H, 0);
    std::vector<uint64_t> row_hash(H, 0);
    std::vector<int64_t> row_kind((size_t)H * 5, 0), row_work((size_t)H * 3, 0);
    parallel_for(H, n_threads(o), [&](int64_t y, int) {
        std::vector<std::vector<int>> cols(W);
        cols_pool(V, o, rows[y], cols);
        std::vector<Cand> cand;
        uint64_t hsum = 0;
        for (int x = 0; x < W; ++x) {
            pixel_candidates(V, o, cols[x], x, (int)y, cand);
            double Mc = std::max({std::fabs(o->bg[0]), std::fabs(o->bg[1]), std::fabs(o->bg[2])}), Mz = 0, dzm = 0;
            for (const Cand& cd : cand) {
                const Geo& G = V.geo[cd.idx];
                Mc = std::max({Mc, G.rgb[0], G.rgb[1], G.rgb[2]});
                Mz = std::max(Mz, std::fabs(G.z));
                dzm = std::max(dzm, cd.dz);
            }
            PixelResult R;
            Compositor comp{V, o, Mc, Mz, dzm, max_branches, &R};
            comp.run(cand, 0, 1.0, 0, 0, 0, 0, 0, true, 0.0, false);
            const int64_t p = y * W + x;
            rgb[p * 3 + 0] = R.primary.r; rgb[p * 3 + 1] = R.primary.g; rgb[p * 3 + 2] = R.primary.b;
            depth[p] = R.primary.d; if (alpha) alpha[p] = R.primary.a;
            if (err_a) err_a[p] = R.primary.ea;
            if (tol_rgb) tol_rgb[p] = R.tol_rgb;
            if (tol_d) tol_d[p] = R.tol_d;
            if (n_alt) n_alt[p] = (int32_t)R.alts.size();
            if (grad_amb) grad_amb[p] = R.grad_amb ? 1 : 0;
            for (auto& L : R.alts) row_alts[y].push_back(L);
            row_amb[y] += R.ambiguous;
            row_wide[y] += R.widened;
            for (int k = 0; k < 5; ++k) row_kind[(size_t)y * 5 + k] += R.amb_kind[k];
            row_work[(size_t)y * 3 + 0] += R.contrib;
            row_work[(size_t)y * 3 + 1] += R.reached;
            row_work[(size_t)y * 3 + 2] += R.terminated;
            hsum += mix(R.hash, (uint64_t)p);
        }
        row_hash[y] = hsum;
    });
    int64_t need = 0, amb = 0, wide = 0; uint64_t h = 0;
    for (int y = 0; y < H; ++y) { need += (int64_t)row_alts[y].size(); amb += row_amb[y]; wide += row_wide[y]; h += row_hash[y]; }
    if (stats) {
        stats[0] = need; stats[1] = amb; std::memcpy(&stats[2], &h, 8); stats[3] = (int64_t)V.geo.size();
        int64_t kind[5] = {0, 0, 0, 0, 0};
        for (int y = 0; y < H; ++y) for (int k = 0; k < 5; ++k) kind[k] += row_kind[(size_t)y * 5 + k];
        for (int k = 0; k < 4; ++k) stats[4 + k] = kind[k];
        for (int k = 0; k < 3; ++k) { int64_t sum = 0; for (int y = 0; y < H; ++y) sum += row_work[(size_t)y * 3 + k]; stats[8 + k] = sum; }
        stats[11] = kind[4];
        stats[12] = wide;
    }
    if (alt && need <= alt_cap) {
        int64_t k = 0;
        for (int y = 0; y < H; ++y) for (auto& L : row_alts[y]) {
            double* q = alt + k * 6;
            q[0] = L.r; q[1] = L.g; q[2] = L.b; q[3] = L.d; q[4] = L.a; q[5] = L.ea; ++k; }
        return 0;
    }
    return need <= alt_cap ? 0 : 1;
}

// Sec. IV (assets fitted by gradient descent on rendered images): adjoint of
// oracle_render_view's primary branch for L = sum grad_rgb . RGB + grad_depth . D.
// Accumulates (+=) into the gradient arrays, which are laid out like the scene arrays
// (g_sh is [G,16,3]; g_pose is [E,K,12]).  The err_* arrays (same layouts, all null or all
// set) receive an FP32 error model of the same gradients: per composited (pixel, Gaussian)
// pair, an absolute error bound of each of its 10 per-instance partials -- from the relative
// bounds of alpha and T of the forward model, the FP32 cancellation in the remainder
// (C_out - P_i) / T_{i+1} (a sum of the pixel's composited terms, (n + 2) u of the colour's
// magnitude, divided by T_{i+1}), the FP32 colour and depth, the centre error bound in the pixel
// offsets, and (P + 32) u of the sum of the partial's magnitudes for its FP32 accumulation over
// the P pixels -- carried through the chain rule one partial at a time and added in absolute
// value.  Returns 0, or -1 on bad arguments.
int oracle_backward_view(const oracle_scene* s, const oracle_opts* o, int e, int c,
                         const double* grad_rgb, const double* grad_depth,
                         double* g_mean, double* g_log_scale, double* g_quat, double* g_logit,
                         double* g_sh, double* g_pose, double* err_mean, double* err_log_scale, double* err_quat,
                         double* err_logit, double* err_sh, double* err_pose) {
    ViewData V;
    if (!build_view(s, o, e, c, V)) return -1;
    std::vector<std::vector<int>> rows;
    row_pools(V, o, rows);
    const int W = V.W, H = V.H;
    const int nth = n_threads(o);
    const size_t NG = V.geo.size();
    const bool want_err = err_mean != nullptr;
    const double u = 5.9604644775390625e-08;
    // Per-instance adjoints: du, dv, da, db, dc, dopac, dr, dg, db, dz (10 per instance); with the
    // error model also their error bounds (10), magnitudes (10) and pixel count (1)
    const size_t NA = want_err ? 31 : 10;
    std::vector<std::vector<double>> acc(nth, std::vector<double>(NG * NA, 0.0));
    parallel_for(H, nth, [&](int64_t y, int tid) {
        std::vector<std::vector<int>> cols(W);
        cols_pool(V, o, rows[y], cols);
        std::vector<Cand> cand;
        std::vector<int> ci; std::vector<double> al, Ti, ex, dTs;
        double* A = acc[tid].data();
        for (int x = 0; x < W; ++x) {
            pixel_candidates(V, o, cols[x], x, (int)y, cand);
            // Primary forward, recording the contributors (and the relative FP32 bound of T before each).
            ci.clear(); al.clear(); Ti.clear(); ex.clear(); dTs.clear();
            double T = 1.0, dT = 0.0, Mc = std::max({std::fabs(o->bg[0]), std::fabs(o->bg[1]), std::fabs(o->bg[2])}),
                   Mz = 0.0;
            for (const Cand& cd : cand) {
                const Geo& G = V.geo[cd.idx];
                if (!G.present || cd.q > o->q_max) continue;
                const double e1 = std::exp(-0.5 * cd.q);
                const double a = std::min(o->alpha_max, G.opac * e1);
                if (a < o->alpha_min) continue;
                const double Tn = T * (1 - a);
                if (Tn < o->t_min) break;
                ci.push_back((int)(&cd - cand.data())); al.push_back(a); Ti.push_back(T); ex.push_back(e1);
                dTs.push_back(dT);
                dT += a / (1 - a) * cd.da + 2 * u;
                Mc = std::max({Mc, G.rgb[0], G.rgb[1], G.rgb[2]});
                Mz = std::max(Mz, std::fabs(G.z));
                T = Tn;
            }
            const int64_t p = y * W + x;
            const double gC[3] = {grad_rgb[p * 3], grad_rgb[p * 3 + 1], grad_rgb[p * 3 + 2]};
            const double gD = grad_depth ? grad_depth[p] : 0.0;
            const double nc = (double)ci.size();
            // Suffix sums behind contributor i (including the background term bg*T_final).
            double S[3] = {o->bg[0] * T, o->bg[1] * T, o->bg[2] * T}, SD = 0;
            for (int n = (int)ci.size() - 1; n >= 0; --n) {
                const Cand& cd = cand[ci[n]];
                const Geo& G = V.geo[cd.idx];
                const double a = al[n], Tb = Ti[n], w = a * Tb, Ta = Tb * (1 - a);
                double* r = A + (size_t)cd.idx * NA;
                // dL/dalpha = T_i [ gC . (rgb_i - S_i/T_{i+1}) + gD (z_i - SD_i/T_{i+1}) ]
                double ga = 0;
                for (int ch = 0; ch < 3; ++ch) ga += gC[ch] * (G.rgb[ch] - S[ch] / Ta);
                ga += gD * (G.z - SD / Ta);
                ga *= Tb;
                double inc[10] = {0, 0, 0, 0, 0, 0, w * gC[0], w * gC[1], w * gC[2], w * gD};
                double err[10] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
                const double dTa = dTs[n] + a / (1 - a) * cd.da + 2 * u;   // relative bound of T after
                if (want_err) {
                    const double ew = std::fabs(w) * (cd.da + dTs[n] + 2 * u);
                    for (int ch = 0; ch < 3; ++ch) err[6 + ch] = ew * std::fabs(gC[ch]);
                    err[9] = ew * std::fabs(gD);
                }
                double e_ga = 0;
                if (want_err) {
                    // remainder (C_out - P_i) / T_{i+1}: FP32 sums of the pixel's composited terms
                    e_ga = std::fabs(ga) * (dTs[n] + 2 * u);
                    for (int ch = 0; ch < 3; ++ch)
                        e_ga += Tb * std::fabs(gC[ch]) * (64 * u * (std::fabs(G.rgb[ch]) + 1.0) + (nc + 2) * u * Mc / Ta +
                                                          std::fabs(S[ch] / Ta) * (dTa + 2 * u));
                    e_ga += Tb * std::fabs(gD) * (G.dz + (nc + 2) * u * Mz / Ta + std::fabs(SD / Ta) * (dTa + 2 * u));
                }
                for (int ch = 0; ch < 3; ++ch) S[ch] += w * G.rgb[ch];
                SD += w * G.z;
                if (!(G.opac * ex[n] > o->alpha_max)) {   // clamped: no gradient to opacity or q
                    inc[5] = ga * ex[n];
                    const double gq = ga * (-0.5 * a);
                    const double dx = cd.dx, dy = cd.dy;           // d = pixel - u
                    const double lx = G.Q[0][0] * dx + G.Q[0][1] * dy, ly = G.Q[0][1] * dx + G.Q[1][1] * dy;
                    inc[2] = gq * dx * dx; inc[3] = gq * 2 * dx * dy; inc[4] = gq * dy * dy;
                    inc[0] = gq * (-2.0) * lx;
                    inc[1] = gq * (-2.0) * ly;
                    if (want_err) {
                        const double e_gq = 0.5 * a * (e_ga + std::fabs(ga) * cd.da);
                        const double du = G.du, dv = G.dv, agq = std::fabs(gq);
                        err[5] = e_ga * ex[n] + std::fabs(ga * ex[n]) * cd.da;
                        err[2] = e_gq * dx * dx + agq * (2 * std::fabs(dx) * du + 4 * u * dx * dx);
                        err[3] = 2 * (e_gq * std::fabs(dx * dy) + agq * (std::fabs(dy) * du + std::fabs(dx) * dv + 4 * u * std::fabs(dx * dy)));
                        err[4] = e_gq * dy * dy + agq * (2 * std::fabs(dy) * dv + 4 * u * dy * dy);
                        err[0] = 2 * (e_gq * std::fabs(lx) + agq * (std::fabs(G.Q[0][0]) * du + std::fabs(G.Q[0][1]) * dv +
                                                                   8 * u * (std::fabs(G.Q[0][0] * dx) + std::fabs(G.Q[0][1] * dy))));
                        err[1] = 2 * (e_gq * std::fabs(ly) + agq * (std::fabs(G.Q[0][1]) * du + std::fabs(G.Q[1][1]) * dv +
                                                                   8 * u * (std::fabs(G.Q[0][1] * dx) + std::fabs(G.Q[1][1] * dy))));
                    }
                }
                for (int k = 0; k < 10; ++k) r[k] += inc[k];
                if (want_err) {
                    for (int k = 0; k < 10; ++k) { r[10 + k] += err[k]; r[20 + k] += std::fabs(inc[k]); }
                    r[30] += 1;
                }
            }
        }
    });
    std::vector<double> tot(NG * NA, 0.0);
    for (int t = 0; t < nth; ++t) for (size_t i = 0; i < NG * NA; ++i) tot[i] += acc[t][i];
    auto add = [&](const InstGrad& q, const Geo& G, double* gm, double* gl, double* gqt, double* go, double* gs,
                   double* gp, bool absval) {
        auto f = [absval](double v) { return absval ? std::fabs(v) : v; };
        const int64_t g = G.g;
        for (int k = 0; k < 3; ++k) { gm[g * 3 + k] += f(q.mean[k]); gl[g * 3 + k] += f(q.log_scale[k]); }
        for (int k = 0; k < 4; ++k) gqt[g * 4 + k] += f(q.quat[k]);
        go[g] += f(q.logit);
        for (int k = 0; k < 48; ++k) gs[g * 48 + k] += f(q.sh[k]);
        double* pp = gp + ((int64_t)e * s->K + G.slot) * 12;
        for (int k = 0; k < 12; ++k) pp[k] += f(q.pose[k]);
    };
    // Chain rule through projection, colour and pose (serial: deterministic accumulation).
    for (size_t i = 0; i < NG; ++i) {
        const Geo& G = V.geo[i];
        const double* r = &tot[i * NA];
        bool any = false; for (int k = 0; k < 10; ++k) any |= r[k] != 0; if (!any) continue;
        InstGrad q;
        chain_rule(s, G, r, q);
        add(q, G, g_mean, g_log_scale, g_quat, g_logit, g_sh, g_pose, false);
        if (!want_err) continue;
        // error bound of each partial: its per-pixel bounds plus its FP32 accumulation over the pixels
        for (int k = 0; k < 10; ++k) {
            double unit[10] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
            unit[k] = r[10 + k] + (r[30] + 32) * u * r[20 + k];
            if (unit[k] == 0) continue;
            InstGrad qk;
            chain_rule(s, G, unit, qk);
            add(qk, G, err_mean, err_log_scale, err_quat, err_logit, err_sh, err_pose, true);
        }
    }
    return 0;
}

}  // extern "C"
