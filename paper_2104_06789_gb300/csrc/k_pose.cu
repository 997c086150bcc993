// Pose-update kernels (Sec. 5.2): Monte-Carlo minimal groups drawn with
// Philox4x64-10, FP64 P3P per group (Eq. 17), order-preserving hypothesis
// collection with se(3) logarithms, and the weighted Gaussian meanshift of
// Eqs. 18-19 on a thread-block cluster.
#include <algorithm>

#include <cooperative_groups.h>

#include "df32.cuh"
#include "voldor_internal.cuh"

namespace cg = cooperative_groups;

namespace vd {

// ---------------------------------------------------------------------------
// FP64 helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ double d3dot(const double* a, const double* b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

__device__ __forceinline__ void d3cross(const double* a, const double* b, double* o)
{
    o[0] = a[1] * b[2] - a[2] * b[1];
    o[1] = a[2] * b[0] - a[0] * b[2];
    o[2] = a[0] * b[1] - a[1] * b[0];
}

__device__ __forceinline__ bool d3unit(double* a)
{
    const double n = sqrt(d3dot(a, a));
    if (!(n > 0.0)) return false;
    const double r = 1.0 / n;
    a[0] *= r; a[1] *= r; a[2] *= r;
    return true;
}

__device__ __forceinline__ double horner4(const double* c, double x)
{
    return (((c[4] * x + c[3]) * x + c[2]) * x + c[1]) * x + c[0];
}

// x = J^-1 F through the adjugate; false if J is singular.
__device__ __forceinline__ bool solve3x3(const double* J, const double* F, double* x)
{
    const double c00 = J[4] * J[8] - J[5] * J[7];
    const double c01 = J[5] * J[6] - J[3] * J[8];
    const double c02 = J[3] * J[7] - J[4] * J[6];
    const double det = J[0] * c00 + J[1] * c01 + J[2] * c02;
    if (!(fabs(det) > 0.0)) return false;
    const double c10 = J[2] * J[7] - J[1] * J[8];
    const double c11 = J[0] * J[8] - J[2] * J[6];
    const double c12 = J[1] * J[6] - J[0] * J[7];
    const double c20 = J[1] * J[5] - J[2] * J[4];
    const double c21 = J[2] * J[3] - J[0] * J[5];
    const double c22 = J[0] * J[4] - J[1] * J[3];
    const double id = 1.0 / det;
    x[0] = (c00 * F[0] + c10 * F[1] + c20 * F[2]) * id;
    x[1] = (c01 * F[0] + c11 * F[1] + c21 * F[2]) * id;
    x[2] = (c02 * F[0] + c12 * F[1] + c22 * F[2]) * id;
    return true;
}

// Largest real root of m^3 + A m^2 + B m + C (Cardano or trigonometric form),
// refined by Newton steps.
__device__ double cubic_max_root(double A, double B, double C)
{
    const double A3 = A / 3.0;
    const double pp = B - A * A3;                         // y^3 + pp y + qq = 0, m = y - A/3
    const double qq = 2.0 * A3 * A3 * A3 - A3 * B + C;
    double y;
    const double disc = 0.25 * qq * qq + pp * pp * pp / 27.0;
    if (disc > 0.0) {
        const double sq = sqrt(disc);
        y = cbrt(-0.5 * qq + sq) + cbrt(-0.5 * qq - sq);
    } else {
        const double r = sqrt(fmax(-pp / 3.0, 0.0));
        double arg = (r > 0.0) ? (-0.5 * qq) / (r * r * r) : 0.0;
        arg = fmin(1.0, fmax(-1.0, arg));
        y = 2.0 * r * cos(acos(arg) / 3.0);
    }
    double m = y - A3;
    for (int it = 0; it < 4; ++it) {
        const double f = ((m + A) * m + B) * m + C;
        const double df = (3.0 * m + 2.0 * A) * m + B;
        if (!(fabs(df) > 0.0)) break;
        const double mn = m - f / df;
        const double fn = ((mn + A) * mn + B) * mn + C;
        if (!(fabs(fn) < fabs(f))) break;
        m = mn;
    }
    return m;
}

// Real root candidates of a quartic (ascending coefficients) by Ferrari's
// method, before polishing, shifted back by -b/4. Returns the count (<= 4).
__device__ int quartic_candidates(const double* a, double* roots)
{
    double amax = 0.0;
    for (int i = 0; i < 4; ++i) amax = fmax(amax, fabs(a[i]));
    if (!(fabs(a[4]) > 1e-14 * amax)) return 0;           // degenerate group
    const double b = a[3] / a[4], c = a[2] / a[4], d = a[1] / a[4], e = a[0] / a[4];
    const double bb = b * b;
    const double P = c - 0.375 * bb;
    const double Q = d - 0.5 * b * c + 0.125 * bb * b;
    const double R = e - 0.25 * b * d + 0.0625 * bb * c - (3.0 / 256.0) * bb * bb;
    double y[4];
    int n = 0;
    // y^4 + P y^2 + Q y + R = (y^2 + P/2 + m)^2 - 2m (y - Q/(4m))^2 for the
    // resolvent root m of m^3 + P m^2 + (P^2/4 - R) m - Q^2/8 = 0
    const double m = cubic_max_root(P, 0.25 * P * P - R, -0.125 * Q * Q);
    if (m > 1e-300 && fabs(Q) > 0.0) {
        const double sr = sqrt(2.0 * m);
        const double h = Q / (2.0 * sr);
        const double c1 = 0.5 * P + m - h, c2 = 0.5 * P + m + h;
        const double D1 = 2.0 * m - 4.0 * c1, D2 = 2.0 * m - 4.0 * c2;
        if (D1 >= 0.0) { const double q = sqrt(D1); y[n++] = 0.5 * (-sr + q); y[n++] = 0.5 * (-sr - q); }
        if (D2 >= 0.0) { const double q = sqrt(D2); y[n++] = 0.5 * (sr + q); y[n++] = 0.5 * (sr - q); }
    } else {
        const double D = P * P - 4.0 * R;                 // biquadratic y^4 + P y^2 + R
        if (D >= 0.0) {
            const double z1 = 0.5 * (-P + sqrt(D)), z2 = 0.5 * (-P - sqrt(D));
            if (z1 >= 0.0) { y[n++] = sqrt(z1); y[n++] = -sqrt(z1); }
            if (z2 >= 0.0) { y[n++] = sqrt(z2); y[n++] = -sqrt(z2); }
        }
    }
    for (int i = 0; i < n; ++i) roots[i] = y[i] - 0.25 * b;
    return n;
}

// One candidate root polished by Newton steps on the quartic.
__device__ double polish_quartic_root(const double* a, double x)
{
    for (int it = 0; it < 3; ++it) {
        const double f = horner4(a, x);
        const double df = ((4.0 * a[4] * x + 3.0 * a[3]) * x + 2.0 * a[2]) * x + a[1];
        if (!(fabs(df) > 0.0)) break;
        const double xn = x - f / df;
        if (!(fabs(horner4(a, xn)) < fabs(f))) break;
        x = xn;
    }
    return x;
}

// Frame spanned by a triangle: f1 along q3 - q1, f3 normal, f2 = f3 x f1
// (columns of F, row-major).
__device__ __forceinline__ bool tri_frame(const double* q1, const double* q2, const double* q3, double* F)
{
    double f1[3] = {q3[0] - q1[0], q3[1] - q1[1], q3[2] - q1[2]};
    const double e[3] = {q2[0] - q1[0], q2[1] - q1[1], q2[2] - q1[2]};
    if (!d3unit(f1)) return false;
    double f3[3];
    d3cross(f1, e, f3);
    if (!d3unit(f3)) return false;
    double f2[3];
    d3cross(f3, f1, f2);
    for (int r = 0; r < 3; ++r) { F[r * 3 + 0] = f1[r]; F[r * 3 + 1] = f2[r]; F[r * 3 + 2] = f3[r]; }
    return true;
}

// ---------------------------------------------------------------------------
// P3P. With s_i the distances along the unit bearings b_i, the law of cosines
// gives s_i^2 + s_k^2 - 2 c_ik s_i s_k = d_ik^2. With u = s2/s1, v = s3/s1:
//   (ii)/(i):  v^2 - 2 c13 v = g(u),  g(u) = (d13/d12)(1 + u^2 - 2 c12 u) - 1
//   with (iii): v D(u) = N(u),  N = d23 (1 + g) - d13 (u^2 + g),
//                               D = 2 d13 (c13 - c23 u)
//   and N^2 - 2 c13 N D - g D^2 = 0 is a quartic in u.
// Each root is polished by Newton steps on the three distance equations; the
// pose maps the world triangle onto the camera triangle. Solutions with all
// s_i > 0 come back sorted by s1.
// ---------------------------------------------------------------------------
struct P3PSol {
    double s1;
    double Rt[12];
};

// The quartic of a P3P instance and the quantities its roots are mapped back
// with. False for a degenerate triangle.
struct P3PSetup {
    double d12, d13, d23, c12, c13, c23;
    double N[3], D[2], Q[5];
};

__device__ bool p3p_setup(const double P[3][3], const double b[3][3], P3PSetup& q)
{
    double e12[3], e13[3], e23[3];
    for (int i = 0; i < 3; ++i) { e12[i] = P[0][i] - P[1][i]; e13[i] = P[0][i] - P[2][i]; e23[i] = P[1][i] - P[2][i]; }
    const double d12 = d3dot(e12, e12), d13 = d3dot(e13, e13), d23 = d3dot(e23, e23);
    if (!(d12 > 0.0 && d13 > 0.0 && d23 > 0.0)) return false;
    const double c12 = d3dot(b[0], b[1]), c13 = d3dot(b[0], b[2]), c23 = d3dot(b[1], b[2]);
    const double K2 = d13 / d12;
    const double g[3] = {K2 - 1.0, -2.0 * K2 * c12, K2};
    q.d12 = d12; q.d13 = d13; q.d23 = d23; q.c12 = c12; q.c13 = c13; q.c23 = c23;
    q.N[0] = (d23 - d13) * g[0] + d23; q.N[1] = (d23 - d13) * g[1]; q.N[2] = (d23 - d13) * g[2] - d13;
    q.D[0] = 2.0 * d13 * c13; q.D[1] = -2.0 * d13 * c23;
    const double* N = q.N;
    const double* D = q.D;
    for (int i = 0; i < 5; ++i) q.Q[i] = 0.0;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) q.Q[i + j] += N[i] * N[j];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 2; ++j) q.Q[i + j] -= 2.0 * c13 * N[i] * D[j];
    const double DD[3] = {D[0] * D[0], 2.0 * D[0] * D[1], D[1] * D[1]};
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) q.Q[i + j] -= g[i] * DD[j];
    return true;
}

// The pose of one polished root u of the quartic: v, the distances s_i
// (polished by Newton steps on the three distance equations), then the
// rotation and translation that map the world triangle onto the camera
// triangle. False if the root gives no solution with all s_i > 0.
__device__ bool p3p_from_root(const double P[3][3], const double b[3][3], const P3PSetup& q, const double u,
                              P3PSol& sol)
{
    const double d12 = q.d12, d13 = q.d13, d23 = q.d23, c12 = q.c12, c13 = q.c13, c23 = q.c23;
    const double* N = q.N;
    const double* D = q.D;
    if (!(u > 0.0)) return false;
    const double Du = D[0] + D[1] * u;
    if (Du == 0.0) return false;
    const double v = (N[0] + (N[1] + N[2] * u) * u) / Du;
    const double q1 = 1.0 + u * u - 2.0 * c12 * u;
    if (!(q1 > 0.0)) return false;
    double s[3];
    s[0] = sqrt(d12 / q1);
    s[1] = u * s[0];
    s[2] = v * s[0];
    if (!(s[0] > 0.0 && s[1] > 0.0 && s[2] > 0.0) || !isfinite(s[2])) return false;
    for (int it = 0; it < 5; ++it) {
        const double F[3] = {s[0] * s[0] + s[1] * s[1] - 2.0 * c12 * s[0] * s[1] - d12,
                             s[0] * s[0] + s[2] * s[2] - 2.0 * c13 * s[0] * s[2] - d13,
                             s[1] * s[1] + s[2] * s[2] - 2.0 * c23 * s[1] * s[2] - d23};
        const double J[9] = {2.0 * (s[0] - c12 * s[1]), 2.0 * (s[1] - c12 * s[0]), 0.0,
                             2.0 * (s[0] - c13 * s[2]), 0.0, 2.0 * (s[2] - c13 * s[0]),
                             0.0, 2.0 * (s[1] - c23 * s[2]), 2.0 * (s[2] - c23 * s[1])};
        double ds[3];
        if (!solve3x3(J, F, ds)) break;
        const double nsv[3] = {s[0] - ds[0], s[1] - ds[1], s[2] - ds[2]};
        const double G0 = nsv[0] * nsv[0] + nsv[1] * nsv[1] - 2.0 * c12 * nsv[0] * nsv[1] - d12;
        const double G1 = nsv[0] * nsv[0] + nsv[2] * nsv[2] - 2.0 * c13 * nsv[0] * nsv[2] - d13;
        const double G2 = nsv[1] * nsv[1] + nsv[2] * nsv[2] - 2.0 * c23 * nsv[1] * nsv[2] - d23;
        if (!(fabs(G0) + fabs(G1) + fabs(G2) < fabs(F[0]) + fabs(F[1]) + fabs(F[2]))) break;
        s[0] = nsv[0]; s[1] = nsv[1]; s[2] = nsv[2];
    }
    if (!(s[0] > 0.0 && s[1] > 0.0 && s[2] > 0.0)) return false;
    double Qc[3][3];
    for (int i = 0; i < 3; ++i)
        for (int c = 0; c < 3; ++c) Qc[i][c] = s[i] * b[i][c];
    double Fw[9], Fc[9];
    if (!tri_frame(P[0], P[1], P[2], Fw) || !tri_frame(Qc[0], Qc[1], Qc[2], Fc)) return false;
    sol.s1 = s[0];
    double cw[3], cc[3];
    for (int c = 0; c < 3; ++c) {
        cw[c] = (P[0][c] + P[1][c] + P[2][c]) / 3.0;
        cc[c] = (Qc[0][c] + Qc[1][c] + Qc[2][c]) / 3.0;
    }
    for (int r0 = 0; r0 < 3; ++r0) {
        for (int c = 0; c < 3; ++c)
            sol.Rt[r0 * 4 + c] = Fc[r0 * 3 + 0] * Fw[c * 3 + 0] + Fc[r0 * 3 + 1] * Fw[c * 3 + 1] + Fc[r0 * 3 + 2] * Fw[c * 3 + 2];
    }
    for (int r0 = 0; r0 < 3; ++r0)
        sol.Rt[r0 * 4 + 3] = cc[r0] - (sol.Rt[r0 * 4 + 0] * cw[0] + sol.Rt[r0 * 4 + 1] * cw[1] + sol.Rt[r0 * 4 + 2] * cw[2]);
    return true;
}

// ---------------------------------------------------------------------------
// Minimal groups of frame t at iteration k (Sec. 5.2): the pixels with a 3D-2D
// correspondence (pi_{t-1} valid), in pixel order, form the list V_t of n
// entries; Philox(index g, t, k, POSE) gives j_i = V_t[hi64(r_i * n)] and a
// group with a repeated pixel yields nothing. P3P (Eq. 17) takes the points in
// camera t-1 and the bearings of the flow targets pi_{t-1} + X_t in camera t,
// all in FP64.
// ---------------------------------------------------------------------------

// The i-th valid pixel of the frame (0 <= i < n): the block whose record
// offset is the last one <= i (the count pass's exclusive scan), then the
// (i - offset)-th set bit of that block's per-warp ballots.
__device__ int valid_pixel_at(const DevState& s, int nb, int i)
{
    int lo = 0, hi = nb - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (s.pix_block_count[mid] <= i) lo = mid;
        else hi = mid - 1;
    }
    int r = i - s.pix_block_count[lo];
    const unsigned* m = s.pix_vmask + (size_t)lo * (kPixThreads / 32);
    for (int w = 0; w < kPixThreads / 32; ++w) {
        unsigned mw = m[w];
        const int c = __popc(mw);
        if (r < c) {
            for (int q = 0; q < r; ++q) mw &= mw - 1u;
            return lo * kPixThreads + w * 32 + (__ffs(mw) - 1);
        }
        r -= c;
    }
    return -1;
}

// Point in camera t-1 and bearing of the flow target of valid pixel j, in
// FP64 (P3P's inputs): P = C_{t-1} theta K^-1 [x y 1], pi_{t-1} its
// projection (the pixel itself for t = 1), the flow X_t sampled bilinearly at
// pi_{t-1}. False if the pixel has no correspondence after all (the pose
// preparation lists it by the same test in float-float; the two can differ
// only within ~1e-11 px of the image border).
__device__ bool group_point(const DevParams& p, const DevState& s, const double* C, int t, int j, double* P,
                            double* bear)
{
    const int x = j % p.W, y = j / p.W;
    const double th = (double)s.theta[j];
    const double d[3] = {((double)x - p.cxd) / p.fxd, ((double)y - p.cyd) / p.fyd, 1.0};
    double u, v;
    if (t == 1) {
        P[0] = th * d[0]; P[1] = th * d[1]; P[2] = th;
        u = x; v = y;
        if (!(P[2] > 0.0)) return false;
    } else {
        const double X = th * d[0], Y = th * d[1], Z = th;
        for (int r = 0; r < 3; ++r) P[r] = C[r * 4 + 0] * X + C[r * 4 + 1] * Y + C[r * 4 + 2] * Z + C[r * 4 + 3];
        if (!(P[2] > 0.0)) return false;
        u = p.fxd * P[0] / P[2] + p.cxd;
        v = p.fyd * P[1] / P[2] + p.cyd;
    }
    if (!(u >= 0.0 && u <= (double)(p.W - 1) && v >= 0.0 && v <= (double)(p.H - 1))) return false;
    const int x0 = min((int)floor(u), p.W - 2), y0 = min((int)floor(v), p.H - 2);
    const double ax = u - x0, ay = v - y0;
    const size_t base = (size_t)(t - 1) * p.N + (size_t)y0 * p.W + x0;
    const float2 f00 = load_flow(s.flows, p.flow_f16, base), f10 = load_flow(s.flows, p.flow_f16, base + 1);
    const float2 f01 = load_flow(s.flows, p.flow_f16, base + p.W), f11 = load_flow(s.flows, p.flow_f16, base + p.W + 1);
    const double w00 = (1 - ax) * (1 - ay), w10 = ax * (1 - ay), w01 = (1 - ax) * ay, w11 = ax * ay;
    const double fu = w00 * f00.x + w10 * f10.x + w01 * f01.x + w11 * f11.x;
    const double fv = w00 * f00.y + w10 * f10.y + w01 * f01.y + w11 * f11.y;
    bear[0] = (u + fu - p.cxd) / p.fxd;
    bear[1] = (v + fv - p.cyd) / p.fyd;
    bear[2] = 1.0;
    return d3unit(bear);
}

// Groups are solved in order in chunks of kP3PChunk (one warp each: four
// lanes per group, one per root of its quartic) until the frame has S
// solutions or the budget of G groups is spent. A warp claims chunks with an
// atomic counter, so the claimed chunks are always 0, 1, ..., c - 1, and every
// claimed chunk is solved: the solved groups form a prefix of the group order.
// After its first chunk a warp claims another only while the solutions found
// so far plus the chunks still in flight, at the yield observed so far, fall
// short of S; the warp that completes the last chunk in flight sees exact
// counts, so the run ends with at least S solutions in the prefix (or the
// whole budget solved), and the first S solutions in group order are the same
// whatever the timing.
//
// Within a quad, lanes 0-2 compute the FP64 point and bearing of the group's
// pixels 0-2 and share them by shuffles; every lane forms the quartic and its
// Ferrari candidates, lane r polishes candidate r and turns it into a pose,
// and each solution's slot is its rank by s1 among the quad's solutions
// (ties by root order): the group's solutions sorted by s1. A warp's
// FP64 dependency chain is then the common part and one root, not up to four
// roots in turn.
constexpr int kP3PChunk = 8;

__global__ void __launch_bounds__(32) k_p3p_groups(DevParams p, DevState s, int t)
{
    const int lane = threadIdx.x, quad = lane >> 2, r = lane & 3, base = lane & ~3;
    const unsigned FULL = 0xffffffffu;
    const int n_valid = *s.pix_count;
    if (n_valid < 3) return;                              // every group repeats a pixel
    const int k = *s.iter;
    const int nb = (p.N + kPixThreads - 1) / kPixThreads;
    const int n_chunks = (p.G + kP3PChunk - 1) / kP3PChunk;
    const double* C = s.cum + 12 * (t - 1);
    bool first = true;
    for (;;) {
        int c = -1;
        if (lane == 0) {
            bool claim = first;
            if (!first) {
                const unsigned long long d = atomicAdd(s.p3p_done, 0ull);
                const long long done = (long long)(d >> 32), sols = (long long)(d & 0xffffffffull);
                const long long inflight = max(0LL, (long long)atomicAdd(s.p3p_claims, 0) - done);
                claim = sols + (done > 0 ? inflight * sols / done : inflight) < (long long)p.S;
            }
            if (claim) c = atomicAdd(s.p3p_claims, 1);
        }
        first = false;
        c = __shfl_sync(FULL, c, 0);
        if (c < 0 || c >= n_chunks) break;
        const int g = c * kP3PChunk + quad;
        const bool active = g < p.G;
        // the group's pixels: j_i = V_t[hi64(r_i n)] (all lanes of the quad draw the same)
        int idx[3] = {0, 0, 0};
        bool distinct = false;
        if (active) {
            const U64x4 rr = philox4x64_10((uint64_t)g, (uint64_t)t, (uint64_t)k, (uint64_t)kStreamPose, p.seed,
                                           p.window_id);
            for (int i = 0; i < 3; ++i) idx[i] = (int)__umul64hi(rr.v[i], (uint64_t)n_valid);
            distinct = idx[0] != idx[1] && idx[0] != idx[2] && idx[1] != idx[2];
        }
        // lane r < 3: pixel r's point in camera t-1 and bearing (FP64)
        double Pm[3] = {0.0, 0.0, 0.0}, bm[3] = {0.0, 0.0, 1.0};
        double wv = 0.0;
        int ok = 1;
        if (active && distinct && r < 3) {
            const int ri = r == 0 ? idx[0] : (r == 1 ? idx[1] : idx[2]);
            const int j = valid_pixel_at(s, nb, ri);
            ok = (j >= 0 && group_point(p, s, C, t, j, Pm, bm)) ? 1 : 0;
            if (ok) wv = (double)s.wmap[(size_t)(t - 1) * p.N + j];
        }
        double P[3][3], b[3][3];
        double weight = 1.0;
        int okall = 1;
#pragma unroll
        for (int i = 0; i < 3; ++i) {
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                P[i][q] = __shfl_sync(FULL, Pm[q], base + i);
                b[i][q] = __shfl_sync(FULL, bm[q], base + i);
            }
            weight *= __shfl_sync(FULL, wv, base + i);
            okall &= __shfl_sync(FULL, ok, base + i);
        }
        const bool valid_group = active && distinct && okall;
        if (!valid_group) weight = 0.0;
        // the quartic (every lane), then lane r's root
        P3PSetup qs;
        int nr = 0;
        double cand[4] = {0.0, 0.0, 0.0, 0.0};
        if (valid_group && p3p_setup(P, b, qs)) nr = quartic_candidates(qs.Q, cand);
        P3PSol sol;
        sol.s1 = 0.0;
        bool has = false;
        if (r < nr) {
            const double u0 = r == 0 ? cand[0] : (r == 1 ? cand[1] : (r == 2 ? cand[2] : cand[3]));
            has = p3p_from_root(P, b, qs, polish_quartic_root(qs.Q, u0), sol);
        }
        // slot = rank by s1 among the quad's solutions, ties by root order
        int rank = 0, cnt = 0;
#pragma unroll
        for (int o = 0; o < 4; ++o) {
            const double so = __shfl_sync(FULL, sol.s1, base + o);
            const int ho = __shfl_sync(FULL, has ? 1 : 0, base + o);
            cnt += ho;
            if (has && ho && (so < sol.s1 || (so == sol.s1 && o < r))) ++rank;
        }
        if (active) {
            if (r == 0) {
                s.grp_count[g] = cnt;
                s.grp_weight[g] = weight;
            }
            if (has) {
                double* o = s.grp_sols + ((size_t)g * kMaxSols + rank) * 12;
                for (int q = 0; q < 12; ++q) o[q] = sol.Rt[q];
            }
        }
        int tot = (r == 0) ? cnt : 0;
        for (int o = 16; o > 0; o >>= 1) tot += __shfl_xor_sync(FULL, tot, o);
        __threadfence();
        if (lane == 0) atomicAdd(s.p3p_done, (1ull << 32) | (unsigned long long)tot);
    }
}

// Groups solved for the current frame (a prefix of the group order).
__device__ __forceinline__ int groups_solved(const DevParams& p, const DevState& s)
{
    const int n_chunks = (p.G + kP3PChunk - 1) / kP3PChunk;
    return min(min(*s.p3p_claims, n_chunks) * kP3PChunk, p.G);
}

// One warp per block spreads the FP64 solves over the SMs. The first wave
// is sized for about 1.1 S solutions at the yield of driving-like windows
// (1.4-1.5 solutions per group); further chunks are claimed as needed.
void launch_p3p_groups(const DevParams& p, const DevState& s, int t, cudaStream_t st)
{
    const int n_chunks = (p.G + kP3PChunk - 1) / kP3PChunk;
    const int wave = std::max(1, std::min(n_chunks, (3 * p.S + 4 * kP3PChunk - 1) / (4 * kP3PChunk)));
    k_p3p_groups<<<wave, 32, 0, st>>>(p, s, t);
}

// ---------------------------------------------------------------------------
// Hypothesis collection: exclusive scan of the group solution counts (one
// block), then one thread per group writes its solutions h = offset + i < S
// with their scoring form and se(3) logarithm.
// ---------------------------------------------------------------------------
__global__ void k_hyp_scan(DevParams p, DevState s)
{
    __shared__ int wsum[32];
    const int tid = threadIdx.x, nt = blockDim.x;
    const int G = groups_solved(p, s);
    const int seg = (G + nt - 1) / nt;
    const int g0 = min(tid * seg, G), g1 = min(g0 + seg, G);
    // segments of a multiple of 4 counts start 16-byte aligned (the arrays are
    // 256-byte aligned): read and write them four at a time
    const bool vec = (seg & 3) == 0;
    const int gv = vec ? g0 + ((g1 - g0) & ~3) : g0;
    int local = 0;
    for (int g = g0; g < gv; g += 4) {
        const int4 c = *reinterpret_cast<const int4*>(s.grp_count + g);
        local += c.x + c.y + c.z + c.w;
    }
    for (int g = gv; g < g1; ++g) local += s.grp_count[g];
    // block exclusive scan of `local`
    const int lane = tid & 31, warp = tid >> 5;
    int incl = local;
    for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += v;
    }
    if (lane == 31) wsum[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        const int nw = nt >> 5;
        int v = lane < nw ? wsum[lane] : 0;
        for (int o = 1; o < 32; o <<= 1) {
            const int u = __shfl_up_sync(0xffffffffu, v, o);
            if (lane >= o) v += u;
        }
        if (lane < nw) wsum[lane] = v;
    }
    __syncthreads();
    int off = incl - local + (warp > 0 ? wsum[warp - 1] : 0);
    for (int g = g0; g < gv; g += 4) {
        const int4 c = *reinterpret_cast<const int4*>(s.grp_count + g);
        int4 o;
        o.x = off; o.y = o.x + c.x; o.z = o.y + c.y; o.w = o.z + c.z;
        *reinterpret_cast<int4*>(s.grp_offset + g) = o;
        off = o.w + c.w;
    }
    for (int g = gv; g < g1; ++g) {
        s.grp_offset[g] = off;
        off += s.grp_count[g];
    }
    if (tid == nt - 1) *s.n_hyp = min(off, p.S);
}

// se(3) logarithm through the unit quaternion of R (Shepperd's selection):
// phi = 2 atan2(|v|, w) v/|v|, rho = V^-1 t with
// V^-1 = I - Phi/2 + (1 - (th/2) cot(th/2)) / th^2 Phi^2, where
// cot(th/2) = w / |v| (w = cos(th/2), |v| = sin(th/2), w >= 0): no FP64
// sine or cosine, which are long serial routines on this GPU's FP64 pipe.
__device__ void se3_log_quat(const double* Rt, double* p6)
{
    const double R00 = Rt[0], R01 = Rt[1], R02 = Rt[2];
    const double R10 = Rt[4], R11 = Rt[5], R12 = Rt[6];
    const double R20 = Rt[8], R21 = Rt[9], R22 = Rt[10];
    const double tr = R00 + R11 + R22;
    double w, x, y, z;
    if (tr >= R00 && tr >= R11 && tr >= R22) {
        w = 0.5 * sqrt(1.0 + tr);
        const double f = 0.25 / w;
        x = (R21 - R12) * f; y = (R02 - R20) * f; z = (R10 - R01) * f;
    } else if (R00 >= R11 && R00 >= R22) {
        x = 0.5 * sqrt(1.0 + R00 - R11 - R22);
        const double f = 0.25 / x;
        w = (R21 - R12) * f; y = (R01 + R10) * f; z = (R02 + R20) * f;
    } else if (R11 >= R22) {
        y = 0.5 * sqrt(1.0 - R00 + R11 - R22);
        const double f = 0.25 / y;
        w = (R02 - R20) * f; x = (R01 + R10) * f; z = (R12 + R21) * f;
    } else {
        z = 0.5 * sqrt(1.0 - R00 - R11 + R22);
        const double f = 0.25 / z;
        w = (R10 - R01) * f; x = (R02 + R20) * f; y = (R12 + R21) * f;
    }
    if (w < 0.0) { w = -w; x = -x; y = -y; z = -z; }
    const double vn = sqrt(x * x + y * y + z * z);
    const double th = 2.0 * atan2(vn, w);
    const double scale = (vn > 1e-8) ? th / vn : (2.0 / w) * (1.0 - vn * vn / (3.0 * w * w));
    const double phi[3] = {scale * x, scale * y, scale * z};
    double c2;
    if (th < 1e-4) c2 = 1.0 / 12.0 + th * th / 720.0;
    else c2 = (1.0 - 0.5 * th * w / vn) / (th * th);
    const double t[3] = {Rt[3], Rt[7], Rt[11]};
    double a[3], b[3];
    d3cross(phi, t, a);
    d3cross(phi, a, b);
    for (int i = 0; i < 3; ++i) p6[i] = t[i] - 0.5 * a[i] + c2 * b[i];
    p6[3] = phi[0]; p6[4] = phi[1]; p6[5] = phi[2];
}

// se(3) exponential: R = I + A Phi + B Phi^2, t = rho + B phi x rho + C phi x (phi x rho).
__device__ void se3_exp_vec(const double* p6, double* Rt)
{
    const double* rho = p6;
    const double* phi = p6 + 3;
    const double th2 = d3dot(phi, phi), th = sqrt(th2);
    double A, B, C;
    if (th < 1e-4) {
        A = 1.0 - th2 / 6.0 + th2 * th2 / 120.0;
        B = 0.5 - th2 / 24.0 + th2 * th2 / 720.0;
        C = 1.0 / 6.0 - th2 / 120.0 + th2 * th2 / 5040.0;
    } else {
        A = sin(th) / th;
        B = (1.0 - cos(th)) / th2;
        C = (th - sin(th)) / (th2 * th);
    }
    const double wx = phi[0], wy = phi[1], wz = phi[2];
    // Phi^2 = phi phi^T - th^2 I
    Rt[0] = 1.0 + B * (wx * wx - th2); Rt[1] = -A * wz + B * wx * wy;       Rt[2] = A * wy + B * wx * wz;
    Rt[4] = A * wz + B * wx * wy;       Rt[5] = 1.0 + B * (wy * wy - th2); Rt[6] = -A * wx + B * wy * wz;
    Rt[8] = -A * wy + B * wx * wz;      Rt[9] = A * wx + B * wy * wz;       Rt[10] = 1.0 + B * (wz * wz - th2);
    double a[3], b[3];
    d3cross(phi, rho, a);
    d3cross(phi, a, b);
    Rt[3] = rho[0] + B * a[0] + C * b[0];
    Rt[7] = rho[1] + B * a[1] + C * b[1];
    Rt[11] = rho[2] + B * a[2] + C * b[2];
}

// One thread per (group, solution slot), so that each thread's FP64 chain is
// a single se(3) logarithm.
__global__ void k_hyp_write(DevParams p, DevState s)
{
    const int gi = blockIdx.x * blockDim.x + threadIdx.x;
    if (gi >= groups_solved(p, s) * kMaxSols) return;
    const int g = gi / kMaxSols, i = gi % kMaxSols;
    if (i >= s.grp_count[g]) return;
    const int h = s.grp_offset[g] + i;
    if (h >= p.S) return;
    const double q = p.fyd / p.fxd;
    const double sc[3] = {1.0, q, 1.0};
    const double* Rt = s.grp_sols + ((size_t)g * kMaxSols + i) * 12;
    double* oR = s.hyp_Rt + (size_t)h * 12;
    for (int r = 0; r < 3; ++r) {
        for (int c = 0; c < 3; ++c) oR[r * 3 + c] = Rt[r * 4 + c];
        oR[9 + r] = Rt[r * 4 + 3];
    }
    float* f = s.hyp_f32 + (size_t)h * 12;
    for (int r = 0; r < 3; ++r) {
        for (int c = 0; c < 3; ++c) f[r * 3 + c] = (float)(sc[r] * (Rt[r * 4 + c] - (r == c ? 1.0 : 0.0)) / sc[c]);
        f[9 + r] = (float)(sc[r] * Rt[r * 4 + 3]);
    }
    s.hyp_w[h] = s.grp_weight[g];
    s.hyp_info[(size_t)h * 2 + 0] = g;
    s.hyp_info[(size_t)h * 2 + 1] = i;
}

// The meanshift's form of hypothesis h (after k_hyp_write): its se(3)
// logarithm, each coordinate as a float-float pair (hi = v rounded, lo =
// v - hi rounded), and its weight in FP32. A long FP64 chain per hypothesis,
// needed only by the meanshift: it runs on a side branch beside the scoring.
__global__ void k_hyp_log(DevParams p, DevState s)
{
    const int h = blockIdx.x * blockDim.x + threadIdx.x;
    if (h >= *s.n_hyp) return;
    const long long g = s.hyp_info[(size_t)h * 2 + 0], i = s.hyp_info[(size_t)h * 2 + 1];
    double pv[6];
    se3_log_quat(s.grp_sols + ((size_t)g * kMaxSols + i) * 12, pv);
    float hi[6], lo[6];
    for (int c = 0; c < 6; ++c) {
        hi[c] = (float)pv[c];
        lo[c] = (float)(pv[c] - (double)hi[c]);
    }
    float4* pw = reinterpret_cast<float4*>(s.hyp_pw + (size_t)h * 16);
    pw[0] = make_float4(hi[0], hi[1], hi[2], hi[3]);
    pw[1] = make_float4(hi[4], hi[5], lo[0], lo[1]);
    pw[2] = make_float4(lo[2], lo[3], lo[4], lo[5]);
    pw[3] = make_float4((float)s.hyp_w[h], 0.f, 0.f, 0.f);
}

void launch_hyp_log(const DevParams& p, const DevState& s, cudaStream_t st)
{
    k_hyp_log<<<(p.S + 127) / 128, 128, 0, st>>>(p, s);
}

void launch_hyp_collect(const DevParams& p, const DevState& s, cudaStream_t st)
{
    k_hyp_scan<<<1, 1024, 0, st>>>(p, s);
    // sized for the budget; threads past the solved prefix return at once
    k_hyp_write<<<(p.G * kMaxSols + 127) / 128, 128, 0, st>>>(p, s);
}

// Scoring form of caller-given hypotheses already copied to hyp_Rt.
__global__ void k_hyp_from_rt(DevParams p, DevState s, int n)
{
    const int h = blockIdx.x * blockDim.x + threadIdx.x;
    if (h == 0) *s.n_hyp = n;
    if (h >= n) return;
    const double q = p.fyd / p.fxd;
    const double sc[3] = {1.0, q, 1.0};
    const double* R = s.hyp_Rt + (size_t)h * 12;
    float* f = s.hyp_f32 + (size_t)h * 12;
    for (int r = 0; r < 3; ++r) {
        for (int c = 0; c < 3; ++c) f[r * 3 + c] = (float)(sc[r] * (R[r * 3 + c] - (r == c ? 1.0 : 0.0)) / sc[c]);
        f[9 + r] = (float)(sc[r] * R[9 + r]);
    }
}

void score_hyps_from_host(const DevParams& p, const DevState& s, int n, cudaStream_t st)
{
    k_hyp_from_rt<<<(n + 127) / 128 + 1, 128, 0, st>>>(p, s, n);
}

// ---------------------------------------------------------------------------
// Meanshift (Eqs. 18-19): x <- sum_h w_h K(x - p_h) p_h / sum_h w_h K(x - p_h),
// K(d) = exp(-d^T Sigma^-1 d / 2), seeded at argmax_h L_h (lowest index on
// ties), on a cluster of kMeanshiftCtas CTAs. Everything runs on the FP32
// pipe (an FP64 instruction is a long issue on this GPU's FP64 pipe, and this
// kernel is a chain of small dependent steps): the argmax compares the FP64
// scores as order-preserving integer keys; each hypothesis is held as its
// FP32 offset from the seed, taken from float-float copies of the se(3)
// logarithms, so the Gaussian and the per-thread partial sums are FP32 on
// small numbers; sums across warps and CTAs and the state (the offset of x
// from the seed) are float-float, about 44 significant bits. Every CTA
// reduces the cluster's partial sums in the same order, so all take the same
// steps; partial buffers alternate by iteration parity so one cluster barrier
// per step suffices, and one warp finishes the step (sums across CTAs, new
// state, convergence) with shuffles. The iteration stops when the step is
// below ms_tol, when a step below 1e-7 no longer contracts (the FP32 noise
// floor of the kernel weights), or after ms_max_iter steps.
// ---------------------------------------------------------------------------
constexpr int kMsCached = 4;     // hypotheses per thread held in registers (all of them up to S = 8192)

__device__ __forceinline__ float warp_sum_f(float v)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Order-preserving integer key of a double: a < b iff key(a) < key(b) for
// non-NaN values, -0 and +0 equal.
__device__ __forceinline__ long long score_key(double v)
{
    long long b = __double_as_longlong(v);
    if (b == (long long)0x8000000000000000ull) b = 0;
    return b >= 0 ? b : (b ^ 0x7fffffffffffffffll);
}

__device__ __forceinline__ DF shfl_df(DF v, int src)
{
    return DF{__shfl_sync(0xffffffffu, v.hi, src), __shfl_sync(0xffffffffu, v.lo, src)};
}

__global__ void __cluster_dims__(kMeanshiftCtas, 1, 1) __launch_bounds__(kMeanshiftThreads, 1)
k_meanshift(DevParams p, DevState s, int t)
{
    cg::cluster_group cluster = cg::this_cluster();
    const unsigned rank = cluster.block_rank();
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarp = blockDim.x >> 5;
    __shared__ float wred[32][8];
    __shared__ float2 part[2][8];
    __shared__ float xo_hi[6], xo_lo[6];      // x - p_seed, float-float
    __shared__ float seed_hi[6], seed_lo[6];
    __shared__ long long bkey[32];
    __shared__ int bidx[32];
    __shared__ int flag;
    const int n = *s.n_hyp;
    if (n == 0) {
        if (rank == 0 && tid == 0) {
            s.status[0] = 0; s.status[1] = -1; s.status[2] = 0; s.status[3] += 1;
        }
        return;   // uniform over the cluster: every CTA reads the same n
    }
    // argmax of L (lowest index on ties; NaN never wins)
    long long bk = 0;
    int bi = 0x7fffffff;
    for (int h = tid; h < n; h += blockDim.x) {
        const double v = s.scores[h];
        const long long raw = __double_as_longlong(v) & 0x7fffffffffffffffll;
        if (raw > 0x7ff0000000000000ll) continue;                 // NaN
        const long long k = score_key(v);
        if (bi == 0x7fffffff || k > bk || (k == bk && h < bi)) { bk = k; bi = h; }
    }
    for (int o = 16; o > 0; o >>= 1) {
        const long long ok = __shfl_xor_sync(0xffffffffu, bk, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (oi != 0x7fffffff && (bi == 0x7fffffff || ok > bk || (ok == bk && oi < bi))) { bk = ok; bi = oi; }
    }
    if (lane == 0) { bkey[warp] = bk; bidx[warp] = bi; }
    __syncthreads();
    if (tid == 0) {
        long long k = bkey[0];
        int i = bidx[0];
        for (int w = 1; w < nwarp; ++w)
            if (bidx[w] != 0x7fffffff && (i == 0x7fffffff || bkey[w] > k || (bkey[w] == k && bidx[w] < i))) {
                k = bkey[w];
                i = bidx[w];
            }
        if (i == 0x7fffffff) i = 0;
        const float* ps = s.hyp_pw + (size_t)i * 16;
        for (int c = 0; c < 6; ++c) {
            seed_hi[c] = ps[c];
            seed_lo[c] = ps[6 + c];
            xo_hi[c] = 0.f;
            xo_lo[c] = 0.f;
        }
        bidx[0] = i;
        flag = 0;
    }
    __syncthreads();
    const int seed = bidx[0];
    // FP32 offsets of this CTA's hypotheses from the seed: a thread's first
    // kMsCached stay in registers, the rest (S above kMsCached x the cluster's
    // threads) go to global memory
    const int stride = kMeanshiftCtas * blockDim.x, h0 = rank * blockDim.x + tid;
    DF sd[6];
    for (int c = 0; c < 6; ++c) sd[c] = DF{seed_hi[c], seed_lo[c]};
    float4 r0[kMsCached], r1[kMsCached];
#pragma unroll
    for (int k = 0; k < kMsCached; ++k) { r0[k] = make_float4(0.f, 0.f, 0.f, 0.f); r1[k] = r0[k]; }
    for (int h = h0, k = 0; h < n; h += stride, ++k) {
        const float4* pw = reinterpret_cast<const float4*>(s.hyp_pw + (size_t)h * 16);
        const float4 a = pw[0], b = pw[1], c2 = pw[2], d = pw[3];
        const float ph[6] = {a.x, a.y, a.z, a.w, b.x, b.y}, pl[6] = {b.z, b.w, c2.x, c2.y, c2.z, c2.w};
        float o[6];
#pragma unroll
        for (int c = 0; c < 6; ++c) o[c] = df_to_float(df_sub(DF{ph[c], pl[c]}, sd[c]));
        const float4 o0 = make_float4(o[0], o[1], o[2], o[3]);
        const float4 o1 = make_float4(o[4], o[5], d.x, 0.f);
        if (k < kMsCached) {
#pragma unroll
            for (int i = 0; i < kMsCached; ++i)
                if (i == k) { r0[i] = o0; r1[i] = o1; }
        } else {
            float4* od = reinterpret_cast<float4*>(s.hyp_dp + (size_t)h * 8);
            od[0] = o0;
            od[1] = o1;
        }
    }
    __shared__ float consts[3];
    if (tid == 0) {
        consts[0] = (float)(1.0 / p.sigma_t);
        consts[1] = (float)(1.0 / p.sigma_r);
        consts[2] = (float)p.ms_tol;
    }
    __syncthreads();
    const float ivt = consts[0], ivr = consts[1], tol = consts[2];
    const float mlog2e = -0.5f * 1.4426950408889634f;
    int it = 0;
    bool degenerate = false;
    float prev_step = INFINITY;
    for (; it < p.ms_max_iter; ++it) {
        float dx[6];
        for (int c = 0; c < 6; ++c) dx[c] = xo_hi[c] + xo_lo[c];
        float acc[7] = {0, 0, 0, 0, 0, 0, 0};
        // hypotheses in increasing h (the registers' first, then global memory)
        auto add = [&](const float4 q0, const float4 q1) {
            const float d0 = dx[0] - q0.x, d1 = dx[1] - q0.y, d2 = dx[2] - q0.z;
            const float d3 = dx[3] - q0.w, d4 = dx[4] - q1.x, d5 = dx[5] - q1.y;
            const float m = fmaf(d0 * d0 + d1 * d1 + d2 * d2, ivt, (d3 * d3 + d4 * d4 + d5 * d5) * ivr);
            const float kw = q1.z * exp2f(mlog2e * m);
            if (!(kw > 0.f)) return;       // zero weight (or a non-finite hypothesis) adds nothing
            acc[0] += kw;
            acc[1] = fmaf(kw, q0.x, acc[1]); acc[2] = fmaf(kw, q0.y, acc[2]); acc[3] = fmaf(kw, q0.z, acc[3]);
            acc[4] = fmaf(kw, q0.w, acc[4]); acc[5] = fmaf(kw, q1.x, acc[5]); acc[6] = fmaf(kw, q1.y, acc[6]);
        };
#pragma unroll
        for (int k = 0; k < kMsCached; ++k)
            if (h0 + k * stride < n) add(r0[k], r1[k]);
        for (int h = h0 + kMsCached * stride; h < n; h += stride) {
            const float4* o = reinterpret_cast<const float4*>(s.hyp_dp + (size_t)h * 8);
            add(o[0], o[1]);
        }
        // warp sums in FP32 (each lane holds at most 4 terms), then the CTA's
        // warps in order as float-float
        float accw[7];
        for (int c = 0; c < 7; ++c) accw[c] = warp_sum_f(acc[c]);
        if (lane == 0)
            for (int c = 0; c < 7; ++c) wred[warp][c] = accw[c];
        __syncthreads();
        const int buf = it & 1;
        if (tid < 7) {
            DF v{0.f, 0.f};
            for (int w = 0; w < nwarp; ++w) v = df_add(v, wred[w][tid]);
            part[buf][tid] = make_float2(v.hi, v.lo);
        }
        cluster.sync();
        if (warp == 0) {
            // entry e = r * 7 + c (component c of rank r's sums, from distributed
            // shared memory) is fetched by lane e % 32 into slot e / 32; lane
            // c < 7 adds the entries of its component in rank order
            static_assert(kMeanshiftCtas * 7 <= 64, "two entries per lane");
            DF g[2] = {DF{0.f, 0.f}, DF{0.f, 0.f}};
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                const int e = lane + 32 * q;
                if (e < kMeanshiftCtas * 7) {
                    const float2 v = *cluster.map_shared_rank(&part[buf][e % 7], (unsigned)(e / 7));
                    g[q] = DF{v.x, v.y};
                }
            }
            DF tot{0.f, 0.f};
            for (int r = 0; r < kMeanshiftCtas; ++r) {
                const int e = r * 7 + (lane < 7 ? lane : 0);
                const DF v0 = shfl_df(g[0], e & 31), v1 = shfl_df(g[1], e & 31);
                tot = df_add(tot, e < 32 ? v0 : v1);
            }
            const DF t0 = shfl_df(tot, 0);
            const bool mass = t0.hi > 0.f;
            float dd = 0.f;
            if (mass && lane >= 1 && lane < 7) {
                const DF xn = df_div(tot, t0);                    // mean offset of component lane - 1
                const DF xo{xo_hi[lane - 1], xo_lo[lane - 1]};
                dd = df_to_float(df_sub(xn, xo));
                dd *= dd;
                xo_hi[lane - 1] = xn.hi;
                xo_lo[lane - 1] = xn.lo;
            }
            float s2 = 0.f;
            for (int c = 1; c < 7; ++c) s2 += __shfl_sync(0xffffffffu, dd, c);
            if (lane == 0) {
                if (!mass) {
                    flag = (it == 0) ? 2 : 1;
                } else {
                    const float step = sqrtf(s2);
                    flag = (step < tol || (step >= prev_step && step < 1e-7f)) ? 1 : 0;
                    prev_step = step;
                }
            }
        }
        __syncthreads();
        const int f = flag;
        if (f == 2) { degenerate = true; break; }
        if (f == 1) { ++it; break; }
    }
    cluster.sync();   // no CTA leaves while another may still read its partials
    if (rank == 0 && tid == 0) {
        s.status[0] = n;
        s.status[1] = seed;
        s.status[2] = it;
        if (degenerate) {
            s.status[3] += 1;
        } else {
            double x[6];
            for (int c = 0; c < 6; ++c)
                x[c] = ((double)seed_hi[c] + (double)seed_lo[c]) + ((double)xo_hi[c] + (double)xo_lo[c]);
            se3_exp_vec(x, s.poses + 12 * (t - 1));
        }
    }
}

void launch_meanshift(const DevParams& p, const DevState& s, int t, cudaStream_t st)
{
    k_meanshift<<<kMeanshiftCtas, kMeanshiftThreads, 0, st>>>(p, s, t);
}

}  // namespace vd
