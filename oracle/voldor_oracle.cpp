// VOLDOR generalized-EM oracle: plain, single-threaded FP64 restatement of the
// inference in "VOLDOR: Visual Odometry from Log-logistic Dense Optical flow
// Residuals" (Min, Yang, Dunn, CVPR 2020).
//
// TEST INFRASTRUCTURE ONLY. Only tests/, __graft_entry__.smoke() and the
// cpu_baseline / reference legs of bench.py may load this library. It shares no
// code, header, table or helper with the CUDA path under
// paper_2104_06789_gb300/csrc, and the product path never calls it.
//
// Every function follows the paper's definitions in the paper's order, with no
// blocking, fusion or reordering. Where the paper is silent the code takes the
// readings listed with each function (the same readings are listed in the
// design notes of the repository).
//
// Parity pins (tests/test_oracle_*.py): Fisk log-pdf against scipy; Philox
// against numpy's Philox4x64-10; forward-backward against brute-force
// enumeration; P3P against the generating pose and a resultant computed by
// sympy; se(3) exp against scipy's matrix exponential; geometry, bilinear
// sampling and triangulation against noiseless synthetic scenes; the full loop
// against the noiseless fixed point and, on a noisy window, against the scale
// equivariance of monocular inference (scale taken from T_1). The paper does
// not fix the noisy trajectory itself: it follows the readings of the
// randomised steps listed with each function.

#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>
#include <algorithm>

extern "C" {

// ---------------------------------------------------------------------------
// Parameters and window state (plain C layout; mirrored by a ctypes Structure).
// ---------------------------------------------------------------------------
typedef struct {
    double a1, a2, b1, b2;        // Fisk parameter functions, Eqs. 5-6
    double lambda_;               // adaptive uniform density, Eq. 7
    double gamma;                 // HMM transition probability, Eq. 11
    double sigma_t, sigma_r;      // pose kernel covariance diagonal (variances), Eq. 18
    double inv_depth_min, inv_depth_max;  // depth sample range (inverse depth)
    double x_min, x_max;          // floor / cap of the squared residual (px^2)
    double beta_min;              // floor of the Fisk shape
    double ms_tol;                // meanshift stop: |dx| < ms_tol
    int hyps_per_frame;           // S: pose hypotheses kept per frame
    int groups_per_frame;         // G: Philox groups drawn per frame (draw budget)
    int ms_max_iter;              // meanshift iteration cap
    int criterion;                // 0: MIE (Eq. 10), 1: MLE (Eq. 9)
    int residual;                 // 0: Fisk (Eqs. 3-6), 1: Gaussian (the ablation's alternative model)
    uint64_t seed, window_id;     // Philox key
} or_params;

typedef struct {
    int width, height, T, pad_;
    double fx, fy, cx, cy;        // pinhole intrinsics K
    or_params p;
    const double* flows;          // [T][H][W][2]: X_t (t = 1..T) at index t-1, on the grid of I_{t-1}
    double* theta;                // [H][W] depth of I_0 (z-depth)
    double* wmap;                 // [T][H][W] unsmoothed rigidness W_t^j
    double* poses;                // [T][16] row-major T_t: camera t-1 -> camera t
} or_window;

enum { OR_OK = 0, OR_DEGENERATE = 5 };
enum { STREAM_POSE = 1, STREAM_DEPTH = 2, STREAM_EPI = 3 };

// ---------------------------------------------------------------------------
// Philox4x64-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy
// as 1, 2, 3", SC'11): 10 rounds of the 4x64 S-box with the key bumped by the
// Weyl constants between rounds.
// ---------------------------------------------------------------------------
void or_philox4x64_10(const uint64_t ctr_in[4], const uint64_t key_in[2], uint64_t out[4])
{
    const uint64_t M0 = 0xD2E7470EE14C6C93ULL, M1 = 0xCA5A826395121157ULL;
    const uint64_t W0 = 0x9E3779B97F4A7C15ULL, W1 = 0xBB67AE8584CAA73BULL;
    uint64_t c[4] = {ctr_in[0], ctr_in[1], ctr_in[2], ctr_in[3]};
    uint64_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) { k0 += W0; k1 += W1; }
        unsigned __int128 p0 = (unsigned __int128)M0 * c[0];
        unsigned __int128 p1 = (unsigned __int128)M1 * c[2];
        uint64_t hi0 = (uint64_t)(p0 >> 64), lo0 = (uint64_t)p0;
        uint64_t hi1 = (uint64_t)(p1 >> 64), lo1 = (uint64_t)p1;
        uint64_t n0 = hi1 ^ c[1] ^ k0;
        uint64_t n1 = lo1;
        uint64_t n2 = hi0 ^ c[3] ^ k1;
        uint64_t n3 = lo0;
        c[0] = n0; c[1] = n1; c[2] = n2; c[3] = n3;
    }
    out[0] = c[0]; out[1] = c[1]; out[2] = c[2]; out[3] = c[3];
}

// Draw the counter (index, t, k, stream) under the window key.
static void draw(const or_window* w, uint64_t index, uint64_t t, uint64_t k, uint64_t stream, uint64_t out[4])
{
    uint64_t ctr[4] = {index, t, k, stream};
    uint64_t key[2] = {w->p.seed, w->p.window_id};
    or_philox4x64_10(ctr, key, out);
}

// Uniform integer in [0, n): high 64 bits of r * n.
static uint64_t scale_index(uint64_t r, uint64_t n)
{
    return (uint64_t)(((unsigned __int128)r * n) >> 64);
}

// Uniform in [0, 1) on the 2^-24 grid (the top 24 bits of the draw).
static double unit24(uint64_t r)
{
    return (double)(r >> 40) * (1.0 / 16777216.0);
}

// ---------------------------------------------------------------------------
// Fisk (log-logistic) residual model, Eqs. 3-7.
// ---------------------------------------------------------------------------

// log of Eq. 4: F(x; alpha, beta) = (beta/alpha)(x/alpha)^(beta-1) / (1 + (x/alpha)^beta)^2
double or_fisk_logpdf(double x, double log_alpha, double beta)
{
    double z = std::log(x) - log_alpha;               // log(x / alpha)
    double bz = beta * z;                              // log((x/alpha)^beta)
    double log1p_pow = bz > 0 ? bz + std::log1p(std::exp(-bz)) : std::log1p(std::exp(bz));
    return std::log(beta) - log_alpha + (beta - 1.0) * z - 2.0 * log1p_pow;
}

// Eqs. 5-6: alpha = a1 exp(a2 |v_ob|), beta = b1 |v_ob| + b2 (floored at beta_min).
void or_fisk_params(const or_params* p, double n, double* log_alpha, double* beta)
{
    *log_alpha = std::log(p->a1) + p->a2 * n;
    *beta = std::max(p->b1 * n + p->b2, p->beta_min);
}

// Gaussian residual model of the ablation study (Sec. 6.3): the 2-D flow
// residual isotropic normal, so the squared EPE x is exponential with mean
// 2 sigma^2. The paper gives no parameters for it; reading: sigma^2(n) is
// matched to the Fisk model at the same flow magnitude by the median of x,
// i.e. 2 sigma^2 ln 2 = alpha(n) (the Fisk median), so
//   log rho = log(ln 2 / alpha) - x ln 2 / alpha.
double or_gauss_logpdf(double x, double log_alpha)
{
    return std::log(std::log(2.0)) - log_alpha - x * std::log(2.0) * std::exp(-log_alpha);
}

static double clamp_x(const or_params* p, double x)
{
    return std::min(std::max(x, p->x_min), p->x_max);
}

// Eq. 10 per-frame term: log[ rho / (rho + mu) ] = -softplus(log mu - log rho).
static double mie_term(double log_rho, double log_mu)
{
    double d = log_mu - log_rho;
    double sp = d > 0 ? d + std::log1p(std::exp(-d)) : std::log1p(std::exp(d));
    return -sp;
}

// Per-(t, j) term of the depth / pose criterion. MIE (Eq. 10): log rho/(rho+mu).
// MLE (Eq. 9): log rho, written as log rho - log mu (mu does not depend on
// the depth or the pose, so the argmax is unchanged). Reading: an invalid
// (t, j) (no observation at pi_{t-1}, or the point behind camera t) takes
// rho := mu, i.e. log 1/2 under MIE and 0 under MLE.
static double crit_term(const or_params* p, bool valid, double log_rho, double log_mu)
{
    if (p->criterion == 1) return valid ? log_rho - log_mu : 0.0;
    return valid ? mie_term(log_rho, log_mu) : std::log(0.5);
}

// ---------------------------------------------------------------------------
// Geometry, Eq. 1.
// ---------------------------------------------------------------------------

// 3x4 rigid transform [R | t] stored row-major in 12 doubles.
static void pose16_to_12(const double* m16, double out[12])
{
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 4; ++c) out[r * 4 + c] = m16[r * 4 + c];
}

static void compose(const double a[12], const double b[12], double out[12])  // a * b
{
    double o[12];
    for (int r = 0; r < 3; ++r) {
        for (int c = 0; c < 3; ++c)
            o[r * 4 + c] = a[r * 4 + 0] * b[0 * 4 + c] + a[r * 4 + 1] * b[1 * 4 + c] + a[r * 4 + 2] * b[2 * 4 + c];
        o[r * 4 + 3] = a[r * 4 + 0] * b[3] + a[r * 4 + 1] * b[7] + a[r * 4 + 2] * b[11] + a[r * 4 + 3];
    }
    std::memcpy(out, o, sizeof(o));
}

static void apply(const double m[12], const double p[3], double out[3])
{
    for (int r = 0; r < 3; ++r)
        out[r] = m[r * 4 + 0] * p[0] + m[r * 4 + 1] * p[1] + m[r * 4 + 2] * p[2] + m[r * 4 + 3];
}

static void identity12(double m[12])
{
    for (int i = 0; i < 12; ++i) m[i] = 0.0;
    m[0] = m[5] = m[10] = 1.0;
}

// Cumulative pose C_t = T_t ... T_1 (C_0 = I): the product of Eq. 1 read with
// T_t the motion from t-1 to t.
static void cumulative(const or_window* w, int t, double C[12])
{
    identity12(C);
    for (int i = 1; i <= t; ++i) {
        double Ti[12];
        pose16_to_12(w->poses + 16 * (i - 1), Ti);
        compose(Ti, C, C);
    }
}

static void project(const or_window* w, const double P[3], double uv[2])
{
    uv[0] = w->fx * P[0] / P[2] + w->cx;
    uv[1] = w->fy * P[1] / P[2] + w->cy;
}

static void backproject(const or_window* w, int x, int y, double depth, double P[3])
{
    P[0] = depth * (x - w->cx) / w->fx;
    P[1] = depth * (y - w->cy) / w->fy;
    P[2] = depth;
}

// Bilinear sample of X_t (t 1-based) at continuous (u, v) on the integer pixel
// grid. Valid iff 0 <= u <= W-1 and 0 <= v <= H-1.
static bool bilinear(const or_window* w, int t, double u, double v, double out[2])
{
    int W = w->width, H = w->height;
    if (!(u >= 0.0 && u <= W - 1 && v >= 0.0 && v <= H - 1)) return false;
    int x0 = std::min((int)std::floor(u), W - 2);
    int y0 = std::min((int)std::floor(v), H - 2);
    double ax = u - x0, ay = v - y0;
    const double* F = w->flows + (size_t)(t - 1) * H * W * 2;
    for (int c = 0; c < 2; ++c) {
        double f00 = F[((size_t)y0 * W + x0) * 2 + c];
        double f10 = F[((size_t)y0 * W + x0 + 1) * 2 + c];
        double f01 = F[((size_t)(y0 + 1) * W + x0) * 2 + c];
        double f11 = F[((size_t)(y0 + 1) * W + x0 + 1) * 2 + c];
        out[c] = (1 - ax) * (1 - ay) * f00 + ax * (1 - ay) * f10 + (1 - ax) * ay * f01 + ax * ay * f11;
    }
    return true;
}

int or_bilinear(const or_window* w, int t, double u, double v, double out[2])
{
    return bilinear(w, t, u, v, out) ? 1 : 0;
}

// One (t, j) evaluation of the mixture model of Eq. 2 at depth `depth`, with
// C_{t-1} and T_t given. Readings: X_t is sampled bilinearly at pi_{t-1}; a
// pixel whose pi_{t-1} leaves the image or lies behind camera t-1 is "invalid
// before" (excluded from P3P groups and from L_h); behind camera t it takes
// rho := mu. The squared residual is floored at x_min and capped at x_max.
struct FrameEval {
    bool valid_prev;   // pi_{t-1} inside the image, P_z > 0 in camera t-1
    bool valid;        // additionally P_z > 0 in camera t
    double P[3];       // point in camera t-1
    double pi_prev[2];
    double vob[2];
    double res[2];     // xi_t - v_ob
    double log_rho, log_mu;
    double ell;        // log rho/(rho+mu); log(1/2) when not valid
    double crit;       // the criterion's term (crit_term)
};

static FrameEval eval_frame(const or_window* w, const double Cprev[12], const double Tt[12],
                            int t, int j, double depth)
{
    FrameEval e;
    std::memset(&e, 0, sizeof(e));
    e.ell = std::log(0.5);
    e.crit = crit_term(&w->p, false, 0.0, 0.0);
    int x = j % w->width, y = j / w->width;
    double P0[3];
    backproject(w, x, y, depth, P0);
    if (t == 1) {
        e.P[0] = P0[0]; e.P[1] = P0[1]; e.P[2] = P0[2];
        e.pi_prev[0] = x; e.pi_prev[1] = y;        // pi_0 is the pixel itself
        if (!(e.P[2] > 0)) return e;
    } else {
        apply(Cprev, P0, e.P);
        if (!(e.P[2] > 0)) return e;
        project(w, e.P, e.pi_prev);
    }
    if (!bilinear(w, t, e.pi_prev[0], e.pi_prev[1], e.vob)) return e;
    e.valid_prev = true;
    double Pt[3];
    apply(Tt, e.P, Pt);
    if (!(Pt[2] > 0)) return e;
    e.valid = true;
    double pi_t[2];
    project(w, Pt, pi_t);
    double xi[2] = {pi_t[0] - e.pi_prev[0], pi_t[1] - e.pi_prev[1]};   // rigid flow
    e.res[0] = xi[0] - e.vob[0];
    e.res[1] = xi[1] - e.vob[1];
    double xsq = clamp_x(&w->p, e.res[0] * e.res[0] + e.res[1] * e.res[1]);
    double n = std::sqrt(e.vob[0] * e.vob[0] + e.vob[1] * e.vob[1]);
    double log_alpha, beta;
    or_fisk_params(&w->p, n, &log_alpha, &beta);
    const double x_mu = clamp_x(&w->p, w->p.lambda_ * w->p.lambda_ * n * n);      // Eq. 7
    if (w->p.residual == 1) {
        e.log_rho = or_gauss_logpdf(xsq, log_alpha);
        e.log_mu = or_gauss_logpdf(x_mu, log_alpha);
    } else {
        e.log_rho = or_fisk_logpdf(xsq, log_alpha, beta);                      // Eq. 3
        e.log_mu = or_fisk_logpdf(x_mu, log_alpha, beta);
    }
    e.ell = mie_term(e.log_rho, e.log_mu);
    e.crit = crit_term(&w->p, true, e.log_rho, e.log_mu);
    return e;
}

static void frame_poses(const or_window* w, int t, double Cprev[12], double Tt[12])
{
    cumulative(w, t - 1, Cprev);
    pose16_to_12(w->poses + 16 * (t - 1), Tt);
}

// ell_t(j) at depth `depth` under the current poses; *valid gets
// (valid_prev ? 1 : 0) + (valid ? 1 : 0).
double or_frame_ell(const or_window* w, int t, int j, double depth, int* valid)
{
    double C[12], Tt[12];
    frame_poses(w, t, C, Tt);
    FrameEval e = eval_frame(w, C, Tt, t, j, depth);
    if (valid) *valid = (e.valid_prev ? 1 : 0) + (e.valid ? 1 : 0);
    return e.ell;
}

// The criterion's term of (t, j) at depth `depth` under the current poses.
double or_frame_crit(const or_window* w, int t, int j, double depth)
{
    double C[12], Tt[12];
    frame_poses(w, t, C, Tt);
    return eval_frame(w, C, Tt, t, j, depth).crit;
}

// Diagnostics of one evaluation: out = {res_u, res_v, pi_prev_u, pi_prev_v,
// vob_u, vob_v, log_rho, log_mu, ell, Px, Py, Pz}.
int or_frame_eval(const or_window* w, int t, int j, double depth, double out[12])
{
    double C[12], Tt[12];
    frame_poses(w, t, C, Tt);
    FrameEval e = eval_frame(w, C, Tt, t, j, depth);
    double o[12] = {e.res[0], e.res[1], e.pi_prev[0], e.pi_prev[1], e.vob[0], e.vob[1],
                    e.log_rho, e.log_mu, e.ell, e.P[0], e.P[1], e.P[2]};
    std::memcpy(out, o, sizeof(o));
    return (e.valid_prev ? 1 : 0) + (e.valid ? 1 : 0);
}

// ---------------------------------------------------------------------------
// Bootstrap (Table 1: W all one; T_1 given; theta triangulated from T_1, X_1).
// Reading: least-squares depth along the ray of pixel j from the two linear
// equations of x_j + X_1^j ~ pi_1(theta); the inverse depth is clamped to
// [inv_depth_min, inv_depth_max], and a non-positive solution is set to the far
// end. T_t for t >= 2 starts at T_1 (used only when a frame has no weighted
// hypothesis).
// ---------------------------------------------------------------------------
void or_bootstrap(or_window* w, const double T1[16])
{
    int W = w->width, H = w->height, T = w->T;
    for (int t = 0; t < T; ++t) std::memcpy(w->poses + 16 * t, T1, 16 * sizeof(double));
    for (size_t i = 0; i < (size_t)T * H * W; ++i) w->wmap[i] = 1.0;
    double M[12];
    pose16_to_12(T1, M);
    for (int y = 0; y < H; ++y) {
        for (int x = 0; x < W; ++x) {
            size_t j = (size_t)y * W + x;
            double d[3] = {(x - w->cx) / w->fx, (y - w->cy) / w->fy, 1.0};
            double Rd[3];
            for (int r = 0; r < 3; ++r) Rd[r] = M[r * 4 + 0] * d[0] + M[r * 4 + 1] * d[1] + M[r * 4 + 2] * d[2];
            const double* f = w->flows + j * 2;
            double mx = (x + f[0] - w->cx) / w->fx;
            double my = (y + f[1] - w->cy) / w->fy;
            // theta * (Rd_x - mx Rd_z) = mx t_z - t_x ; same for y
            double ax = Rd[0] - mx * Rd[2], bx = mx * M[11] - M[3];
            double ay = Rd[1] - my * Rd[2], by = my * M[11] - M[7];
            double num = ax * ax + ay * ay;    // inverse depth = (a.a)/(a.b)
            double den = ax * bx + ay * by;
            double inv = w->p.inv_depth_min;
            if (den > 0 && std::isfinite(num / den))
                inv = std::min(std::max(num / den, w->p.inv_depth_min), w->p.inv_depth_max);
            w->theta[j] = 1.0 / inv;
        }
    }
}

// ---------------------------------------------------------------------------
// P3P (Eq. 17). The paper uses AP3P; every exact P3P solver returns the same
// (at most four) poses. This oracle takes the classical route of Grunert: the
// three law-of-cosines equations in the distances s_i along the bearings,
// reduced with u = s2/s1, v = s3/s1 to a quartic in v. Its real roots are
// bracketed by the real roots of its derivatives and bisected to the last
// representable double. The pose follows from the two congruent triangles.
// Solutions (s_i > 0) are returned sorted by s1.
// ---------------------------------------------------------------------------

// Solves the 3x3 system M x = y by Cramer's rule.
static void solve3(const double M[9], const double y[3], double x[3])
{
    double det = M[0] * (M[4] * M[8] - M[5] * M[7]) - M[1] * (M[3] * M[8] - M[5] * M[6]) + M[2] * (M[3] * M[7] - M[4] * M[6]);
    for (int c = 0; c < 3; ++c) {
        double A[9];
        std::memcpy(A, M, sizeof(A));
        for (int r = 0; r < 3; ++r) A[r * 3 + c] = y[r];
        x[c] = (A[0] * (A[4] * A[8] - A[5] * A[7]) - A[1] * (A[3] * A[8] - A[5] * A[6]) + A[2] * (A[3] * A[7] - A[4] * A[6])) / det;
    }
}

// Polynomials as ascending coefficient vectors.
typedef std::vector<double> Poly;

static Poly padd(const Poly& a, const Poly& b)
{
    Poly r(std::max(a.size(), b.size()), 0.0);
    for (size_t i = 0; i < a.size(); ++i) r[i] += a[i];
    for (size_t i = 0; i < b.size(); ++i) r[i] += b[i];
    return r;
}

static Poly pmul(const Poly& a, const Poly& b)
{
    Poly r(a.size() + b.size() - 1, 0.0);
    for (size_t i = 0; i < a.size(); ++i)
        for (size_t j = 0; j < b.size(); ++j) r[i + j] += a[i] * b[j];
    return r;
}

static Poly pscale(const Poly& a, double s)
{
    Poly r(a);
    for (double& c : r) c *= s;
    return r;
}

static double peval(const Poly& a, double x)
{
    double r = 0.0;
    for (size_t i = a.size(); i-- > 0;) r = r * x + a[i];
    return r;
}

static Poly pderiv(const Poly& a)
{
    if (a.size() <= 1) return Poly(1, 0.0);
    Poly r(a.size() - 1);
    for (size_t i = 1; i < a.size(); ++i) r[i - 1] = a[i] * (double)i;
    return r;
}

static Poly ptrim(Poly a)
{
    while (a.size() > 1 && a.back() == 0.0) a.pop_back();
    return a;
}

// Bisection between lo and hi (f(lo), f(hi) of opposite sign) until no double
// lies strictly between them.
static double bisect(const Poly& a, double lo, double hi)
{
    double flo = peval(a, lo);
    for (int it = 0; it < 4000; ++it) {
        double mid = 0.5 * (lo + hi);
        if (mid <= lo || mid >= hi) break;
        double fm = peval(a, mid);
        if (fm == 0.0) return mid;
        if ((fm < 0) == (flo < 0)) { lo = mid; flo = fm; } else { hi = mid; }
    }
    return std::fabs(peval(a, lo)) <= std::fabs(peval(a, hi)) ? lo : hi;
}

// All real roots of a in [lo, hi] (sorted), found between the real roots of
// its derivative.
static std::vector<double> real_roots(const Poly& a_in, double lo, double hi)
{
    Poly a = ptrim(a_in);
    std::vector<double> roots;
    int n = (int)a.size() - 1;
    if (n <= 0) return roots;
    if (n == 1) {
        double r = -a[0] / a[1];
        if (r >= lo && r <= hi) roots.push_back(r);
        return roots;
    }
    std::vector<double> crit = real_roots(pderiv(a), lo, hi);
    std::vector<double> brk;
    brk.push_back(lo);
    for (double c : crit) if (c > brk.back()) brk.push_back(c);
    if (hi > brk.back()) brk.push_back(hi);
    for (size_t i = 0; i + 1 < brk.size(); ++i) {
        double fa = peval(a, brk[i]), fb = peval(a, brk[i + 1]);
        if (fa == 0.0) {
            if (roots.empty() || roots.back() != brk[i]) roots.push_back(brk[i]);
            continue;
        }
        if ((fa < 0) != (fb < 0) && fb != 0.0) roots.push_back(bisect(a, brk[i], brk[i + 1]));
    }
    double fh = peval(a, brk.back());
    if (fh == 0.0 && (roots.empty() || roots.back() != brk.back())) roots.push_back(brk.back());
    return roots;
}

static double dot3(const double a[3], const double b[3]) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
static void sub3(const double a[3], const double b[3], double o[3]) { o[0] = a[0] - b[0]; o[1] = a[1] - b[1]; o[2] = a[2] - b[2]; }
static void cross3(const double a[3], const double b[3], double o[3])
{
    o[0] = a[1] * b[2] - a[2] * b[1];
    o[1] = a[2] * b[0] - a[0] * b[2];
    o[2] = a[0] * b[1] - a[1] * b[0];
}
static bool normalize3(double a[3])
{
    double n = std::sqrt(dot3(a, a));
    if (!(n > 0)) return false;
    a[0] /= n; a[1] /= n; a[2] /= n;
    return true;
}

// Orthonormal frame of a triangle: e1 along p2-p1, e3 normal, e2 = e3 x e1.
static bool triad(const double p1[3], const double p2[3], const double p3[3], double E[9])
{
    double e1[3], v[3], e3[3], e2[3];
    sub3(p2, p1, e1);
    if (!normalize3(e1)) return false;
    sub3(p3, p1, v);
    cross3(e1, v, e3);
    if (!normalize3(e3)) return false;
    cross3(e3, e1, e2);
    for (int r = 0; r < 3; ++r) { E[r * 3 + 0] = e1[r]; E[r * 3 + 1] = e2[r]; E[r * 3 + 2] = e3[r]; }
    return true;
}

// P: 3 world points (camera t-1), b: 3 unit bearings (camera t), row-major
// [i][xyz]. Outputs up to 4 solutions: Rs[4][9], ts[4][3], s1[4]. Returns the
// count.
int or_p3p(const double P[9], const double b[9], double Rs[36], double ts[12], double s1_out[4])
{
    const double *P1 = P, *P2 = P + 3, *P3 = P + 6;
    const double *b1 = b, *b2 = b + 3, *b3 = b + 6;
    double t12[3], t13[3], t23[3];
    sub3(P1, P2, t12); sub3(P1, P3, t13); sub3(P2, P3, t23);
    double d12 = dot3(t12, t12), d13 = dot3(t13, t13), d23 = dot3(t23, t23);   // squared distances
    double c12 = dot3(b1, b2), c13 = dot3(b1, b3), c23 = dot3(b2, b3);
    if (!(d12 > 0 && d13 > 0 && d23 > 0)) return 0;
    // s1^2 (1 + u^2 - 2u c12) = d12   (i)
    // s1^2 (1 + v^2 - 2v c13) = d13   (ii)
    // s1^2 (u^2 + v^2 - 2uv c23) = d23 (iii)
    // (i)/(ii): u^2 - 2 c12 u = f(v),  f(v) = (d12/d13)(1 + v^2 - 2 v c13) - 1
    // with (iii): u D(v) = N(v), N = d23 (1 + f) - d12 (f + v^2), D = 2 d12 (c12 - c23 v)
    // and N^2 - 2 c12 N D - f D^2 = 0 is the quartic in v.
    double K1 = d12 / d13;
    Poly one_v = {1.0, -2.0 * c13, 1.0};                 // 1 + v^2 - 2 v c13
    Poly f = padd(pscale(one_v, K1), Poly{-1.0});
    Poly vsq = {0.0, 0.0, 1.0};
    Poly N = padd(pscale(padd(Poly{1.0}, f), d23), pscale(padd(f, vsq), -d12));
    Poly D = {2.0 * d12 * c12, -2.0 * d12 * c23};
    Poly Q = padd(padd(pmul(N, N), pscale(pmul(N, D), -2.0 * c12)), pscale(pmul(f, pmul(D, D)), -1.0));
    Q = ptrim(Q);
    double amax = 0.0;
    for (size_t i = 0; i + 1 < Q.size(); ++i) amax = std::max(amax, std::fabs(Q[i]));
    double lead = std::fabs(Q.back());
    if (!(lead > 0)) return 0;
    double bound = 1.0 + amax / lead;                    // Cauchy bound on |root|
    std::vector<double> vs = real_roots(Q, 0.0, bound);
    struct Sol { double s1; double R[9]; double t[3]; };
    std::vector<Sol> sols;
    for (double v : vs) {
        if (!(v > 0)) continue;
        double Dv = peval(D, v);
        if (Dv == 0.0) continue;
        double u = peval(N, v) / Dv;
        double q2 = peval(one_v, v);
        if (!(q2 > 0)) continue;
        double s1 = std::sqrt(d13 / q2);
        double s2 = u * s1, s3 = v * s1;
        if (!(s1 > 0 && s2 > 0 && s3 > 0) || !std::isfinite(s2)) continue;
        // Newton steps on the three law-of-cosines equations themselves; a step
        // is kept only if it lowers the residual.
        for (int it = 0; it < 5; ++it) {
            double F[3] = {s1 * s1 + s2 * s2 - 2 * c12 * s1 * s2 - d12,
                           s1 * s1 + s3 * s3 - 2 * c13 * s1 * s3 - d13,
                           s2 * s2 + s3 * s3 - 2 * c23 * s2 * s3 - d23};
            double J[9] = {2 * s1 - 2 * c12 * s2, 2 * s2 - 2 * c12 * s1, 0.0,
                           2 * s1 - 2 * c13 * s3, 0.0, 2 * s3 - 2 * c13 * s1,
                           0.0, 2 * s2 - 2 * c23 * s3, 2 * s3 - 2 * c23 * s2};
            double det = J[0] * (J[4] * J[8] - J[5] * J[7]) - J[1] * (J[3] * J[8] - J[5] * J[6]) + J[2] * (J[3] * J[7] - J[4] * J[6]);
            if (!(std::fabs(det) > 0)) break;
            double ds[3];
            solve3(J, F, ds);
            double n1 = s1 - ds[0], n2 = s2 - ds[1], n3 = s3 - ds[2];
            double G[3] = {n1 * n1 + n2 * n2 - 2 * c12 * n1 * n2 - d12,
                           n1 * n1 + n3 * n3 - 2 * c13 * n1 * n3 - d13,
                           n2 * n2 + n3 * n3 - 2 * c23 * n2 * n3 - d23};
            if (!(std::fabs(G[0]) + std::fabs(G[1]) + std::fabs(G[2]) < std::fabs(F[0]) + std::fabs(F[1]) + std::fabs(F[2])))
                break;
            s1 = n1; s2 = n2; s3 = n3;
        }
        if (!(s1 > 0 && s2 > 0 && s3 > 0)) continue;
        double Q1[3] = {s1 * b1[0], s1 * b1[1], s1 * b1[2]};
        double Q2[3] = {s2 * b2[0], s2 * b2[1], s2 * b2[2]};
        double Q3[3] = {s3 * b3[0], s3 * b3[1], s3 * b3[2]};
        double Ew[9], Ec[9];
        if (!triad(P1, P2, P3, Ew) || !triad(Q1, Q2, Q3, Ec)) continue;
        Sol s;
        s.s1 = s1;
        // R = Ec Ew^T maps the world triad onto the camera triad; t = Q1 - R P1.
        for (int r = 0; r < 3; ++r)
            for (int c = 0; c < 3; ++c)
                s.R[r * 3 + c] = Ec[r * 3 + 0] * Ew[c * 3 + 0] + Ec[r * 3 + 1] * Ew[c * 3 + 1] + Ec[r * 3 + 2] * Ew[c * 3 + 2];
        for (int r = 0; r < 3; ++r)
            s.t[r] = Q1[r] - (s.R[r * 3 + 0] * P1[0] + s.R[r * 3 + 1] * P1[1] + s.R[r * 3 + 2] * P1[2]);
        sols.push_back(s);
    }
    std::stable_sort(sols.begin(), sols.end(), [](const Sol& a, const Sol& b) { return a.s1 < b.s1; });
    int n = std::min((int)sols.size(), 4);
    for (int i = 0; i < n; ++i) {
        std::memcpy(Rs + 9 * i, sols[i].R, 9 * sizeof(double));
        std::memcpy(ts + 3 * i, sols[i].t, 3 * sizeof(double));
        if (s1_out) s1_out[i] = sols[i].s1;
    }
    return n;
}

// ---------------------------------------------------------------------------
// Monte-Carlo minimal groups (Sec. 5.2, Eqs. 15-17, 19). The paper forms a
// group around a depth-map position that has a 3D-2D correspondence at frame t
// and two further distinct positions; Fig. 6 ties every correspondence to a
// minimal instance. Reading: the positions with a correspondence at frame t
// (pi_{t-1} inside I_{t-1} and P_z > 0 in camera t-1) are listed in pixel
// order, V_t = (v_0 < ... < v_{n-1}); group g of frame t at iteration k draws
// Philox(index g, t, k, POSE) and takes j_i = V_t[hi64(r_i * n)] for
// i = 0, 1, 2; a group with a repeated position yields nothing. Groups
// g = 0, 1, ... are solved in order and their solutions (sorted by s1) are
// appended until S hypotheses exist, drawing at most G groups (the budget).
// The weight of a hypothesis is the product of the unsmoothed W_t of its
// three pixels (Eq. 19).
// ---------------------------------------------------------------------------
static bool has_correspondence(const or_window* w, const double Cprev[12], const double Tt[12], int t, int64_t j)
{
    return eval_frame(w, Cprev, Tt, t, (int)j, w->theta[j]).valid_prev;
}

// Writes V_t (pixel indices in increasing order) into out (room for H*W
// entries) and returns n.
int64_t or_valid_pixels(const or_window* w, int t, int64_t* out)
{
    double C[12], Tt[12];
    frame_poses(w, t, C, Tt);
    int64_t N = (int64_t)w->width * w->height, n = 0;
    for (int64_t j = 0; j < N; ++j)
        if (has_correspondence(w, C, Tt, t, j)) out[n++] = j;
    return n;
}

int or_draw_group(const or_window* w, int k, int t, int64_t g, const int64_t* valid, int64_t n_valid,
                  int64_t j_out[3])
{
    if (n_valid < 1) return 0;
    uint64_t r[4];
    draw(w, (uint64_t)g, (uint64_t)t, (uint64_t)k, STREAM_POSE, r);
    for (int i = 0; i < 3; ++i) j_out[i] = valid[scale_index(r[i], (uint64_t)n_valid)];
    return (j_out[0] != j_out[1] && j_out[0] != j_out[2] && j_out[1] != j_out[2]) ? 1 : 0;
}

// Builds the P3P instance of a group (3D points in camera t-1, bearings of the
// flow targets pi_{t-1} + X_t in camera t). Returns 0 for an invalid group.
static int group_instance(const or_window* w, const double Cprev[12], const double Tt[12], int t,
                          const int64_t j[3], double P[9], double b[9], double* weight)
{
    double wt = 1.0;
    for (int i = 0; i < 3; ++i) {
        FrameEval e = eval_frame(w, Cprev, Tt, t, (int)j[i], w->theta[j[i]]);
        if (!e.valid_prev) return 0;
        double target[2] = {e.pi_prev[0] + e.vob[0], e.pi_prev[1] + e.vob[1]};
        double v[3] = {(target[0] - w->cx) / w->fx, (target[1] - w->cy) / w->fy, 1.0};
        normalize3(v);
        for (int c = 0; c < 3; ++c) { P[i * 3 + c] = e.P[c]; b[i * 3 + c] = v[c]; }
        wt *= w->wmap[(size_t)(t - 1) * w->width * w->height + j[i]];
    }
    *weight = wt;
    return 1;
}

// Collects up to S hypotheses of frame t at iteration k. Outputs (row-major):
// R[S][9], tv[S][3], weight[S], group[S], slot[S]. Returns the count.
int or_collect_hypotheses(const or_window* w, int k, int t, double* R, double* tv, double* weight,
                          int64_t* group, int* slot)
{
    double C[12], Tt[12];
    frame_poses(w, t, C, Tt);
    std::vector<int64_t> valid((size_t)w->width * w->height);
    const int64_t n_valid = or_valid_pixels(w, t, valid.data());
    int S = w->p.hyps_per_frame, G = w->p.groups_per_frame;
    int n = 0;
    for (int64_t g = 0; g < G && n < S; ++g) {
        int64_t j[3];
        if (!or_draw_group(w, k, t, g, valid.data(), n_valid, j)) continue;
        double P[9], b[9], wt;
        if (!group_instance(w, C, Tt, t, j, P, b, &wt)) continue;
        double Rs[36], ts[12], s1[4];
        int m = or_p3p(P, b, Rs, ts, s1);
        for (int i = 0; i < m && n < S; ++i, ++n) {
            std::memcpy(R + 9 * n, Rs + 9 * i, 9 * sizeof(double));
            std::memcpy(tv + 3 * n, ts + 3 * i, 3 * sizeof(double));
            weight[n] = wt;
            group[n] = g;
            slot[n] = i;
        }
    }
    return n;
}

// ---------------------------------------------------------------------------
// Dense hypothesis scoring: L_h = sum_j [valid_prev] W_t^j log[rho/(rho+mu)]
// with T_t = h, i.e. the criterion of Eq. 10 moved onto the pose.
// ---------------------------------------------------------------------------
void or_score_hypotheses(const or_window* w, int t, int n, const double* R, const double* tv, double* L)
{
    double C[12];
    cumulative(w, t - 1, C);
    size_t Np = (size_t)w->width * w->height;
    const double* Wt = w->wmap + (size_t)(t - 1) * Np;
    for (int h = 0; h < n; ++h) {
        double Th[12];
        for (int r = 0; r < 3; ++r) {
            for (int c = 0; c < 3; ++c) Th[r * 4 + c] = R[9 * h + r * 3 + c];
            Th[r * 4 + 3] = tv[3 * h + r];
        }
        double sum = 0.0;
        for (size_t j = 0; j < Np; ++j) {
            FrameEval e = eval_frame(w, C, Th, t, (int)j, w->theta[j]);
            if (!e.valid_prev) continue;
            sum += Wt[j] * e.crit;
        }
        L[h] = sum;
    }
}

// ---------------------------------------------------------------------------
// se(3) exponential and logarithm; p = (rho, phi) with the translation part
// first, t = V(phi) rho.
// ---------------------------------------------------------------------------
static void hat(const double w[3], double M[9])
{
    M[0] = 0; M[1] = -w[2]; M[2] = w[1];
    M[3] = w[2]; M[4] = 0; M[5] = -w[0];
    M[6] = -w[1]; M[7] = w[0]; M[8] = 0;
}

static void mat3mul(const double A[9], const double B[9], double C[9])
{
    double O[9];
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) O[r * 3 + c] = A[r * 3] * B[c] + A[r * 3 + 1] * B[3 + c] + A[r * 3 + 2] * B[6 + c];
    std::memcpy(C, O, sizeof(O));
}

// Coefficients A = sin(th)/th, B = (1-cos th)/th^2, Cc = (th - sin th)/th^3,
// by their Taylor series near 0.
static void exp_coeffs(double th, double* A, double* B, double* Cc)
{
    double t2 = th * th;
    if (th < 1e-4) {
        *A = 1.0 - t2 / 6.0 + t2 * t2 / 120.0;
        *B = 0.5 - t2 / 24.0 + t2 * t2 / 720.0;
        *Cc = 1.0 / 6.0 - t2 / 120.0 + t2 * t2 / 5040.0;
    } else {
        *A = std::sin(th) / th;
        *B = (1.0 - std::cos(th)) / t2;
        *Cc = (th - std::sin(th)) / (t2 * th);
    }
}

void or_se3_exp(const double p[6], double R[9], double t[3])
{
    const double* rho = p;
    const double* phi = p + 3;
    double th = std::sqrt(dot3(phi, phi));
    double A, B, Cc;
    exp_coeffs(th, &A, &B, &Cc);
    double K[9], K2[9];
    hat(phi, K);
    mat3mul(K, K, K2);
    double V[9];
    for (int i = 0; i < 9; ++i) {
        double I = (i % 4 == 0) ? 1.0 : 0.0;
        R[i] = I + A * K[i] + B * K2[i];
        V[i] = I + B * K[i] + Cc * K2[i];
    }
    for (int r = 0; r < 3; ++r) t[r] = V[r * 3] * rho[0] + V[r * 3 + 1] * rho[1] + V[r * 3 + 2] * rho[2];
}


void or_se3_log(const double R[9], const double t[3], double p[6])
{
    // R = I + sin(th) K + (1 - cos th) K^2 with K = [a]x, |a| = 1:
    // R - R^T = 2 sin(th) K and (R + R^T)/2 - cos(th) I = (1 - cos th) a a^T.
    double c = 0.5 * (R[0] + R[4] + R[8] - 1.0);
    double vee[3] = {R[7] - R[5], R[2] - R[6], R[3] - R[1]};    // 2 sin(th) a
    double s = 0.5 * std::sqrt(dot3(vee, vee));
    double th = std::atan2(s, c);
    double phi[3];
    if (th < 1e-4) {
        double f = 0.5 * (1.0 + th * th / 6.0);                 // th / (2 sin th)
        for (int i = 0; i < 3; ++i) phi[i] = f * vee[i];
    } else if (th < M_PI - 1e-2) {
        double f = th / (2.0 * s);
        for (int i = 0; i < 3; ++i) phi[i] = f * vee[i];
    } else {
        double S[9];
        for (int r = 0; r < 3; ++r)
            for (int k = 0; k < 3; ++k)
                S[r * 3 + k] = (0.5 * (R[r * 3 + k] + R[k * 3 + r]) - (r == k ? c : 0.0)) / (1.0 - c);
        int col = 0;
        if (S[4] > S[col * 4]) col = 1;
        if (S[8] > S[col * 4]) col = 2;
        double a[3] = {S[0 * 3 + col], S[1 * 3 + col], S[2 * 3 + col]};
        normalize3(a);
        if (dot3(a, vee) < 0) { a[0] = -a[0]; a[1] = -a[1]; a[2] = -a[2]; }
        for (int i = 0; i < 3; ++i) phi[i] = th * a[i];
    }
    double thp = std::sqrt(dot3(phi, phi));
    double A, B, Cc;
    exp_coeffs(thp, &A, &B, &Cc);
    double K[9], K2[9], V[9];
    hat(phi, K);
    mat3mul(K, K, K2);
    for (int i = 0; i < 9; ++i) V[i] = ((i % 4 == 0) ? 1.0 : 0.0) + B * K[i] + Cc * K2[i];
    double rho[3];
    solve3(V, t, rho);
    p[0] = rho[0]; p[1] = rho[1]; p[2] = rho[2];
    p[3] = phi[0]; p[4] = phi[1]; p[5] = phi[2];
}

// ---------------------------------------------------------------------------
// Weighted Gaussian meanshift on se(3) 6-vectors (Eqs. 18-19, Fig. 6):
// x <- sum_h w_h K(x - p_h) p_h / sum_h w_h K(x - p_h),
// K(d) = exp(-1/2 d^T Sigma^-1 d), Sigma = diag(sigma_t x3, sigma_r x3).
// Starts at p[seed]; stops when |dx| < tol or after max_iter steps. Returns the
// number of steps, or -1 when the kernel mass is zero at the start.
// ---------------------------------------------------------------------------
int or_meanshift(const double* p, const double* wgt, int n, int seed, double sigma_t, double sigma_r,
                 int max_iter, double tol, double x_out[6])
{
    double x[6];
    for (int i = 0; i < 6; ++i) x[i] = p[6 * seed + i];
    int it = 0;
    for (; it < max_iter; ++it) {
        double num[6] = {0, 0, 0, 0, 0, 0}, den = 0.0;
        for (int h = 0; h < n; ++h) {
            double m = 0.0;
            for (int i = 0; i < 6; ++i) {
                double d = x[i] - p[6 * h + i];
                m += d * d / (i < 3 ? sigma_t : sigma_r);
            }
            double k = wgt[h] * std::exp(-0.5 * m);
            den += k;
            for (int i = 0; i < 6; ++i) num[i] += k * p[6 * h + i];
        }
        if (!(den > 0)) {
            if (it == 0) return -1;
            break;
        }
        double step = 0.0;
        for (int i = 0; i < 6; ++i) {
            double xn = num[i] / den;
            step += (xn - x[i]) * (xn - x[i]);
            x[i] = xn;
        }
        if (std::sqrt(step) < tol) { ++it; break; }
    }
    for (int i = 0; i < 6; ++i) x_out[i] = x[i];
    return it;
}

// ---------------------------------------------------------------------------
// Pose update of frame t (Table 1 inner loop; Eqs. 15-19). The meanshift is
// seeded at the hypothesis with the largest dense score L_h (lowest index on
// ties). With no hypothesis, or zero kernel mass, T_t keeps its value and the
// call reports OR_DEGENERATE.
// Optional outputs (may be NULL): n_hyp, L (S), seed index, meanshift steps.
// ---------------------------------------------------------------------------
int or_pose_update(or_window* w, int k, int t, int* n_hyp_out, double* L_out, int* seed_out, int* iters_out)
{
    int S = w->p.hyps_per_frame;
    std::vector<double> R(9 * (size_t)S), tv(3 * (size_t)S), wt(S), L(S), p(6 * (size_t)S);
    std::vector<int64_t> grp(S);
    std::vector<int> slot(S);
    int n = or_collect_hypotheses(w, k, t, R.data(), tv.data(), wt.data(), grp.data(), slot.data());
    if (n_hyp_out) *n_hyp_out = n;
    if (n == 0) return OR_DEGENERATE;
    or_score_hypotheses(w, t, n, R.data(), tv.data(), L.data());
    int seed = 0;
    for (int h = 1; h < n; ++h) if (L[h] > L[seed]) seed = h;
    if (L_out) std::memcpy(L_out, L.data(), n * sizeof(double));
    if (seed_out) *seed_out = seed;
    for (int h = 0; h < n; ++h) or_se3_log(R.data() + 9 * h, tv.data() + 3 * h, p.data() + 6 * h);
    double x[6];
    int its = or_meanshift(p.data(), wt.data(), n, seed, w->p.sigma_t, w->p.sigma_r, w->p.ms_max_iter, w->p.ms_tol, x);
    if (iters_out) *iters_out = its;
    if (its < 0) return OR_DEGENERATE;
    double Rn[9], tn[3];
    or_se3_exp(x, Rn, tn);
    double* M = w->poses + 16 * (t - 1);
    for (int r = 0; r < 3; ++r) {
        for (int c = 0; c < 3; ++c) M[r * 4 + c] = Rn[r * 3 + c];
        M[r * 4 + 3] = tn[r];
    }
    M[12] = 0; M[13] = 0; M[14] = 0; M[15] = 1;
    return OR_OK;
}

// ---------------------------------------------------------------------------
// E-step (Eqs. 11-14). Emission of (t, j) at the current depth and poses,
// normalised: w = rho/(rho+mu) (1/2 where the model takes rho := mu).
// ---------------------------------------------------------------------------
void or_emissions(const or_window* w, double* out)
{
    size_t Np = (size_t)w->width * w->height;
    for (int t = 1; t <= w->T; ++t) {
        double C[12], Tt[12];
        frame_poses(w, t, C, Tt);
        for (size_t j = 0; j < Np; ++j) {
            FrameEval e = eval_frame(w, C, Tt, t, (int)j, w->theta[j]);
            out[(size_t)(t - 1) * Np + j] = std::exp(e.ell);
        }
    }
}

// Forward-backward on one chain of length L with emissions (1-w_j, w_j) for
// (W=0, W=1), transition [[g, 1-g], [1-g, g]], uniform initial state and
// m_b = 1 at the chain end. Messages are normalised at every step. Output:
// q_j = q(W_j = 1).
void or_forward_backward(const double* w, int L, double gamma, double* q)
{
    if (L <= 0) return;
    std::vector<double> f0(L), f1(L), b0(L), b1(L);
    {
        double a0 = 0.5 * (1.0 - w[0]), a1 = 0.5 * w[0], s = a0 + a1;
        f0[0] = a0 / s; f1[0] = a1 / s;
    }
    for (int j = 1; j < L; ++j) {   // Eq. 13
        double p0 = gamma * f0[j - 1] + (1.0 - gamma) * f1[j - 1];
        double p1 = (1.0 - gamma) * f0[j - 1] + gamma * f1[j - 1];
        double a0 = (1.0 - w[j]) * p0, a1 = w[j] * p1, s = a0 + a1;
        f0[j] = a0 / s; f1[j] = a1 / s;
    }
    b0[L - 1] = 1.0; b1[L - 1] = 1.0;
    for (int j = L - 2; j >= 0; --j) {   // Eq. 14
        double e0 = (1.0 - w[j + 1]) * b0[j + 1], e1 = w[j + 1] * b1[j + 1];
        double c0 = gamma * e0 + (1.0 - gamma) * e1;
        double c1 = (1.0 - gamma) * e0 + gamma * e1;
        double s = c0 + c1;
        b0[j] = c0 / s; b1[j] = c1 / s;
    }
    for (int j = 0; j < L; ++j) {   // Eq. 12
        double a0 = f0[j] * b0[j], a1 = f1[j] * b1[j];
        q[j] = a1 / (a0 + a1);
    }
}

// Smooths every W_t along rows (axis 0) or columns (axis 1).
void or_smooth(const or_window* w, int axis, const double* emis, double* q)
{
    int W = w->width, H = w->height;
    size_t Np = (size_t)W * H;
    for (int t = 0; t < w->T; ++t) {
        const double* e = emis + t * Np;
        double* o = q + t * Np;
        if (axis == 0) {
            for (int y = 0; y < H; ++y) or_forward_backward(e + (size_t)y * W, W, w->p.gamma, o + (size_t)y * W);
        } else {
            std::vector<double> ce(H), co(H);
            for (int x = 0; x < W; ++x) {
                for (int y = 0; y < H; ++y) ce[y] = e[(size_t)y * W + x];
                or_forward_backward(ce.data(), H, w->p.gamma, co.data());
                for (int y = 0; y < H; ++y) o[(size_t)y * W + x] = co[y];
            }
        }
    }
}

// ---------------------------------------------------------------------------
// M-step: MIE depth by sampling-propagation on directed 1-D chains (Eq. 10,
// Fig. 5). Readings: one sweep per iteration, direction [L->R, T->B, R->L,
// B->T][k mod 4]; candidates prev (depth before the sweep), nbr (the winner at
// the previous chain pixel; none at the chain start) and smp (uniform in
// inverse depth from Philox(index j, 0, k, DEPTH)); a candidate replaces the
// current best only by a strictly larger score, in the order prev, nbr, smp;
// NaN scores count as -inf.
// ---------------------------------------------------------------------------
static double mie_score(const or_window* w, const std::vector<double>& C, const std::vector<double>& Tt,
                        const double* q, int j, double depth)
{
    size_t Np = (size_t)w->width * w->height;
    double s = 0.0;
    for (int t = 1; t <= w->T; ++t) {
        FrameEval e = eval_frame(w, &C[12 * (t - 1)], &Tt[12 * (t - 1)], t, j, depth);
        s += q[(size_t)(t - 1) * Np + j] * e.crit;
    }
    return std::isnan(s) ? -INFINITY : s;
}

static void all_frame_poses(const or_window* w, std::vector<double>& C, std::vector<double>& Tt)
{
    C.assign(12 * (size_t)w->T, 0.0);
    Tt.assign(12 * (size_t)w->T, 0.0);
    for (int t = 1; t <= w->T; ++t) frame_poses(w, t, &C[12 * (t - 1)], &Tt[12 * (t - 1)]);
}

double or_mie_score(const or_window* w, const double* q, int j, double depth)
{
    std::vector<double> C, Tt;
    all_frame_poses(w, C, Tt);
    return mie_score(w, C, Tt, q, j, depth);
}

double or_depth_sample(const or_window* w, int k, int64_t j)
{
    uint64_t r[4];
    draw(w, (uint64_t)j, 0, (uint64_t)k, STREAM_DEPTH, r);
    double u = unit24(r[0]);
    return 1.0 / (w->p.inv_depth_min + u * (w->p.inv_depth_max - w->p.inv_depth_min));
}

// Chain geometry of direction dir: number of chains, chain length, and pixel
// index of position i of chain c.
static void chain_shape(const or_window* w, int dir, int* n_chains, int* len)
{
    if (dir == 0 || dir == 2) { *n_chains = w->height; *len = w->width; }
    else { *n_chains = w->width; *len = w->height; }
}

static int chain_pixel(const or_window* w, int dir, int c, int i)
{
    int W = w->width, H = w->height;
    switch (dir) {
        case 0: return c * W + i;                 // left to right along row c
        case 1: return i * W + c;                 // top to bottom along column c
        case 2: return c * W + (W - 1 - i);       // right to left
        default: return (H - 1 - i) * W + c;      // bottom to top
    }
}

// labels (may be NULL): 0 prev, 1 nbr, 2 smp.
void or_mie_sweep(or_window* w, int k, const double* q, unsigned char* labels)
{
    std::vector<double> C, Tt;
    all_frame_poses(w, C, Tt);
    size_t Np = (size_t)w->width * w->height;
    std::vector<double> prev(w->theta, w->theta + Np);
    int dir = k % 4, n_chains, len;
    chain_shape(w, dir, &n_chains, &len);
    for (int c = 0; c < n_chains; ++c) {
        int last = -1;
        for (int i = 0; i < len; ++i) {
            int j = chain_pixel(w, dir, c, i);
            double best = prev[j];
            double best_score = mie_score(w, C, Tt, q, j, best);
            unsigned char lab = 0;
            if (last >= 0) {
                double nbr = w->theta[last];
                double s = mie_score(w, C, Tt, q, j, nbr);
                if (s > best_score) { best = nbr; best_score = s; lab = 1; }
            }
            double smp = or_depth_sample(w, k, j);
            double s = mie_score(w, C, Tt, q, j, smp);
            if (s > best_score) { best = smp; best_score = s; lab = 2; }
            w->theta[j] = best;
            if (labels) labels[j] = lab;
            last = j;
        }
    }
}

// Unsmoothed rigidness update (Table 1, last line): W_t^j = rho/(rho+mu).
void or_rigidness(or_window* w)
{
    or_emissions(w, w->wmap);
}

// ---------------------------------------------------------------------------
// One iteration of the VOLDOR loop (Table 1). Returns OR_DEGENERATE if a frame
// kept its previous pose.
// ---------------------------------------------------------------------------
int or_em_iteration(or_window* w, int k)
{
    int status = OR_OK;
    for (int t = 1; t <= w->T; ++t) {
        int s = or_pose_update(w, k, t, nullptr, nullptr, nullptr, nullptr);
        if (s != OR_OK) status = s;
    }
    size_t n = (size_t)w->T * w->width * w->height;
    std::vector<double> emis(n), q(n);
    or_emissions(w, emis.data());
    int dir = k % 4;
    or_smooth(w, (dir == 0 || dir == 2) ? 0 : 1, emis.data(), q.data());
    or_mie_sweep(w, k, q.data(), nullptr);
    or_rigidness(w);
    return status;
}

int or_run(or_window* w, int k0, int n_iters)
{
    int status = OR_OK;
    for (int i = 0; i < n_iters; ++i) {
        int s = or_em_iteration(w, k0 + i);
        if (s != OR_OK) status = s;
    }
    return status;
}


// ---------------------------------------------------------------------------
// Epipolar bootstrap of T_1 (Sec. 5.3 and Table 1: T_1 from the epipolar
// geometry of X_1 by least median of squares, Rousseeuw 1984). Readings:
//  - correspondences m0 = K^-1 [x, y, 1], m1 = K^-1 [x + u, y + v, 1] of every
//    pixel whose flow target lies inside I_1 (0 <= x + u <= W - 1, same for y);
//  - sample m takes 8 pixels j_i = hi64(r_i * N), r_0..3 from the Philox counter
//    (m, 0, 0, EPI) and r_4..7 from (m, 1, 0, EPI); a sample with a repeated or
//    invalid pixel, or whose 8 x 9 system has no one-dimensional null space,
//    scores +inf;
//  - E spans the null space of the 8 x 9 matrix with rows m1 (x) m0 (so that
//    m1^T E m0 = 0; the eigenvector of A^T A of the smallest eigenvalue), then
//    projected onto the essential matrices, E = U diag(1, 1, 0) V^T;
//  - the error of pixel j is Sampson's first-order distance
//    (m1^T E m0)^2 / ((E m0)_1^2 + (E m0)_2^2 + (E^T m1)_1^2 + (E^T m1)_2^2)
//    in calibrated coordinates;
//  - a sample's score is the lower median (rank floor((n - 1) / 2) in ascending
//    order) of the errors of the n valid pixels; the smallest score wins, the
//    lowest sample index on ties;
//  - reweighted least squares after the LMedS fit (Rousseeuw and Leroy 1987):
//    robust scale s = 1.4826 (1 + 5 / (n - 8)) sqrt(median); the pixels whose
//    error under the winning sample is at most (2.5 s)^2 are inliers, and E is
//    re-estimated as the null vector (smallest right singular vector) of the
//    matrix of their rows m1 (x) m0, then projected again (if there are fewer
//    than 8 inliers the sample's E is kept);
//  - (R, t) is the candidate among (U W V^T, +u3), (U W V^T, -u3),
//    (U W^T V^T, +u3), (U W^T V^T, -u3) (det U = det V = +1,
//    W = [[0,-1,0],[1,0,0],[0,0,1]]) with the most valid pixels whose depth,
//    triangulated as in the bootstrap, is positive in both cameras (the first
//    in that order on ties); |t| is set to the caller's baseline (the scale of
//    a monocular window is free).
// ---------------------------------------------------------------------------

// One-sided Jacobi SVD (Hestenes 1958; Golub and Van Loan, Sec. 8.6.4) of an
// m x n matrix A (row-major, overwritten): rotations of column pairs until all
// columns are orthogonal; then A = (A V) V^T with the columns of A V
// orthogonal, their norms the singular values sv[n], V (n x n, row-major) the
// right singular vectors as columns. Works on A itself, so the accuracy of the
// small singular vectors is not squared away as in A^T A.
static void jacobi_svd(double* A, int m, int n, double* sv, double* V)
{
    for (int i = 0; i < n * n; ++i) V[i] = 0.0;
    for (int i = 0; i < n; ++i) V[i * n + i] = 1.0;
    for (int sweep = 0; sweep < 60; ++sweep) {
        bool rotated = false;
        for (int p = 0; p < n - 1; ++p) {
            for (int q = p + 1; q < n; ++q) {
                double alpha = 0.0, beta = 0.0, gamma = 0.0;
                for (int k = 0; k < m; ++k) {
                    alpha += A[k * n + p] * A[k * n + p];
                    beta += A[k * n + q] * A[k * n + q];
                    gamma += A[k * n + p] * A[k * n + q];
                }
                if (!(std::fabs(gamma) > 1e-17 * std::sqrt(alpha * beta))) continue;
                rotated = true;
                const double zeta = (beta - alpha) / (2.0 * gamma);
                const double t = (zeta >= 0 ? 1.0 : -1.0) / (std::fabs(zeta) + std::sqrt(1.0 + zeta * zeta));
                const double c = 1.0 / std::sqrt(1.0 + t * t), s = c * t;
                for (int k = 0; k < m; ++k) {
                    const double ap = A[k * n + p], aq = A[k * n + q];
                    A[k * n + p] = c * ap - s * aq;
                    A[k * n + q] = s * ap + c * aq;
                }
                for (int k = 0; k < n; ++k) {
                    const double vp = V[k * n + p], vq = V[k * n + q];
                    V[k * n + p] = c * vp - s * vq;
                    V[k * n + q] = s * vp + c * vq;
                }
            }
        }
        if (!rotated) break;
    }
    for (int j = 0; j < n; ++j) {
        double s = 0.0;
        for (int k = 0; k < m; ++k) s += A[k * n + j] * A[k * n + j];
        sv[j] = std::sqrt(s);
    }
}

// The 8-point estimate: E (row-major) spans the null space of the 8 x 9 matrix
// with rows m1 (x) m0. Returns 0 if the null space is not one-dimensional.
int or_essential_8pt(const double* m0, const double* m1, double E[9])
{
    // A padded with a zero row to 9 x 9 (the null space is unchanged)
    double A[9 * 9] = {0};
    for (int i = 0; i < 8; ++i)
        for (int r = 0; r < 3; ++r)
            for (int c = 0; c < 3; ++c) A[i * 9 + r * 3 + c] = m1[i * 3 + r] * m0[i * 3 + c];
    double sv[9], V[81];
    jacobi_svd(A, 9, 9, sv, V);
    int order[9];
    for (int i = 0; i < 9; ++i) order[i] = i;
    std::sort(order, order + 9, [&](int a, int b) { return sv[a] < sv[b]; });
    const double smax = sv[order[8]];
    if (!(smax > 0.0) || !(sv[order[1]] > 1e-10 * smax)) return 0;
    for (int k = 0; k < 9; ++k) E[k] = V[k * 9 + order[0]];
    return 1;
}

// SVD of a 3 x 3 matrix: M = U diag(s) V^T with s descending and
// det U = det V = +1 (the third singular pair is fixed by the cross products,
// which the essential projection does not use). Returns 0 if rank(M) < 2.
static int svd3_rank2(const double M[9], double U[9], double s[3], double V[9])
{
    double A[9], sv[3], Q[9];
    std::memcpy(A, M, sizeof(A));
    jacobi_svd(A, 3, 3, sv, Q);
    int o[3] = {0, 1, 2};
    std::sort(o, o + 3, [&](int a, int b) { return sv[a] > sv[b]; });
    double v[3][3], u[3][3];
    for (int i = 0; i < 3; ++i)
        for (int k = 0; k < 3; ++k) v[i][k] = Q[k * 3 + o[i]];
    cross3(v[0], v[1], v[2]);                     // right-handed V
    for (int i = 0; i < 2; ++i) {
        s[i] = sv[o[i]];
        if (!(s[i] > 0.0)) return 0;
        for (int r = 0; r < 3; ++r) u[i][r] = A[r * 3 + o[i]] / s[i];   // columns of M V
    }
    s[2] = sv[o[2]];
    cross3(u[0], u[1], u[2]);
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) { U[r * 3 + c] = u[c][r]; V[r * 3 + c] = v[c][r]; }
    return 1;
}

// Closest essential matrix: U diag(1, 1, 0) V^T. Returns 0 if rank(E) < 2.
int or_essential_project(const double Ein[9], double E[9], double U[9], double V[9])
{
    double s[3];
    if (!svd3_rank2(Ein, U, s, V)) return 0;
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) E[r * 3 + c] = U[r * 3 + 0] * V[c * 3 + 0] + U[r * 3 + 1] * V[c * 3 + 1];
    return 1;
}

double or_sampson(const double E[9], const double m0[3], const double m1[3])
{
    double Em0[3], Etm1[3];
    for (int r = 0; r < 3; ++r) Em0[r] = E[r * 3 + 0] * m0[0] + E[r * 3 + 1] * m0[1] + E[r * 3 + 2] * m0[2];
    for (int c = 0; c < 3; ++c) Etm1[c] = E[0 * 3 + c] * m1[0] + E[1 * 3 + c] * m1[1] + E[2 * 3 + c] * m1[2];
    const double e = m1[0] * Em0[0] + m1[1] * Em0[1] + m1[2] * Em0[2];
    const double den = Em0[0] * Em0[0] + Em0[1] * Em0[1] + Etm1[0] * Etm1[0] + Etm1[1] * Etm1[1];
    if (!(den > 0.0)) return INFINITY;
    return e * e / den;
}

// The four (R, t) of an essential matrix with SVD factors U, V (det +1), in the
// candidate order of the readings; R row-major [4][9], t [4][3] (unit).
void or_essential_candidates(const double U[9], const double V[9], double* R, double* t)
{
    const double Wm[9] = {0, -1, 0, 1, 0, 0, 0, 0, 1};
    for (int a = 0; a < 2; ++a) {
        double UW[9];
        for (int r = 0; r < 3; ++r)
            for (int c = 0; c < 3; ++c) {
                double s = 0.0;
                for (int k = 0; k < 3; ++k) s += U[r * 3 + k] * (a == 0 ? Wm[k * 3 + c] : Wm[c * 3 + k]);
                UW[r * 3 + c] = s;
            }
        double Ra[9];
        for (int r = 0; r < 3; ++r)
            for (int c = 0; c < 3; ++c)
                Ra[r * 3 + c] = UW[r * 3 + 0] * V[c * 3 + 0] + UW[r * 3 + 1] * V[c * 3 + 1] + UW[r * 3 + 2] * V[c * 3 + 2];
        for (int sgn = 0; sgn < 2; ++sgn) {
            const int i = 2 * a + sgn;
            std::memcpy(R + 9 * i, Ra, sizeof(Ra));
            for (int r = 0; r < 3; ++r) t[3 * i + r] = (sgn == 0 ? 1.0 : -1.0) * U[r * 3 + 2];
        }
    }
}

// Correspondence of pixel j: false if the flow target leaves I_1.
static bool epi_corr(const or_window* w, size_t j, double m0[3], double m1[3])
{
    const int x = (int)(j % w->width), y = (int)(j / w->width);
    const double* f = w->flows + j * 2;
    const double u = x + f[0], v = y + f[1];
    if (!(u >= 0.0 && u <= w->width - 1 && v >= 0.0 && v <= w->height - 1)) return false;
    m0[0] = (x - w->cx) / w->fx; m0[1] = (y - w->cy) / w->fy; m0[2] = 1.0;
    m1[0] = (u - w->cx) / w->fx; m1[1] = (v - w->cy) / w->fy; m1[2] = 1.0;
    return true;
}

// Essential matrix of sample m (0 if the sample is invalid).
int or_epi_sample(const or_window* w, int m, double E[9], int64_t j_out[8])
{
    const uint64_t N = (uint64_t)w->width * w->height;
    uint64_t r[8];
    draw(w, (uint64_t)m, 0, 0, STREAM_EPI, r);
    draw(w, (uint64_t)m, 1, 0, STREAM_EPI, r + 4);
    int64_t j[8];
    for (int i = 0; i < 8; ++i) j[i] = (int64_t)scale_index(r[i], N);
    if (j_out) std::memcpy(j_out, j, sizeof(j));
    for (int a = 0; a < 8; ++a)
        for (int b = a + 1; b < 8; ++b)
            if (j[a] == j[b]) return 0;
    double m0[24], m1[24];
    for (int i = 0; i < 8; ++i)
        if (!epi_corr(w, (size_t)j[i], m0 + 3 * i, m1 + 3 * i)) return 0;
    double E8[9], U[9], V[9];
    if (!or_essential_8pt(m0, m1, E8)) return 0;
    return or_essential_project(E8, E, U, V);
}

// Lower median of the Sampson errors of every valid pixel under E.
double or_epi_score(const or_window* w, const double E[9])
{
    std::vector<double> d;
    const size_t N = (size_t)w->width * w->height;
    for (size_t j = 0; j < N; ++j) {
        double m0[3], m1[3];
        if (!epi_corr(w, j, m0, m1)) continue;
        d.push_back(or_sampson(E, m0, m1));
    }
    if (d.empty()) return INFINITY;
    const size_t k = (d.size() - 1) / 2;
    std::nth_element(d.begin(), d.begin() + k, d.end());
    return d[k];
}

// Valid pixels in front of both cameras under (R, t).
int64_t or_epi_cheirality(const or_window* w, const double R[9], const double t[3])
{
    int64_t count = 0;
    const size_t N = (size_t)w->width * w->height;
    for (size_t j = 0; j < N; ++j) {
        double m0[3], m1[3];
        if (!epi_corr(w, j, m0, m1)) continue;
        double Rd[3];
        for (int r = 0; r < 3; ++r) Rd[r] = R[r * 3 + 0] * m0[0] + R[r * 3 + 1] * m0[1] + R[r * 3 + 2] * m0[2];
        // the bootstrap's least-squares depth: z0 = (a.b)/(a.a)
        const double ax = Rd[0] - m1[0] * Rd[2], bx = m1[0] * t[2] - t[0];
        const double ay = Rd[1] - m1[1] * Rd[2], by = m1[1] * t[2] - t[1];
        const double aa = ax * ax + ay * ay, ab = ax * bx + ay * by;
        if (!(aa > 0.0) || !(ab > 0.0)) continue;
        const double z0 = ab / aa;
        const double z1 = z0 * Rd[2] + t[2];
        if (z1 > 0.0) ++count;
    }
    return count;
}

// Number of valid pixels (targets inside I_1).
static int64_t epi_valid_count(const or_window* w)
{
    int64_t n = 0;
    const size_t N = (size_t)w->width * w->height;
    for (size_t j = 0; j < N; ++j) {
        double m0[3], m1[3];
        n += epi_corr(w, j, m0, m1) ? 1 : 0;
    }
    return n;
}

// Reweighted least squares after LMedS: E_out from the inliers of E at the
// given median; returns the inlier count (E_out = E if it is below 8).
int64_t or_epi_refine(const or_window* w, const double E[9], double median, double E_out[9], double* thresh_out)
{
    const int64_t n = epi_valid_count(w);
    std::memcpy(E_out, E, 9 * sizeof(double));
    if (n <= 8) return 0;
    const double s = 1.4826 * (1.0 + 5.0 / (double)(n - 8)) * std::sqrt(median);
    const double thr = (2.5 * s) * (2.5 * s);
    if (thresh_out) *thresh_out = thr;
    std::vector<double> A;
    const size_t N = (size_t)w->width * w->height;
    for (size_t j = 0; j < N; ++j) {
        double m0[3], m1[3];
        if (!epi_corr(w, j, m0, m1) || !(or_sampson(E, m0, m1) <= thr)) continue;
        for (int r = 0; r < 3; ++r)
            for (int c = 0; c < 3; ++c) A.push_back(m1[r] * m0[c]);
    }
    const int64_t n_in = (int64_t)(A.size() / 9);
    if (n_in < 8) return n_in;
    double sv[9], V[81];
    jacobi_svd(A.data(), (int)n_in, 9, sv, V);
    int k0 = 0;
    for (int k = 1; k < 9; ++k)
        if (sv[k] < sv[k0]) k0 = k;
    double En[9], U[9], Vv[9];
    for (int k = 0; k < 9; ++k) En[k] = V[k * 9 + k0];
    if (or_essential_project(En, E_out, U, Vv)) return n_in;
    std::memcpy(E_out, E, 9 * sizeof(double));
    return n_in;
}

// The whole epipolar bootstrap: T_1 (row-major 4 x 4) into T1_out and the
// window state as or_bootstrap leaves it. scores[n_samples] (may be null) gets
// every sample's score. Returns OR_DEGENERATE (state untouched) if no sample is
// valid.
int or_epipolar_bootstrap(or_window* w, int n_samples, double baseline, double T1_out[16], double* scores,
                          int* chosen_out, int* candidate_out)
{
    int best = -1;
    double best_score = INFINITY, bestE[9] = {0};
    for (int m = 0; m < n_samples; ++m) {
        double E[9];
        double s = INFINITY;
        if (or_epi_sample(w, m, E, nullptr)) s = or_epi_score(w, E);
        if (scores) scores[m] = s;
        if (s < best_score) { best_score = s; best = m; std::memcpy(bestE, E, sizeof(E)); }
    }
    if (chosen_out) *chosen_out = best;
    if (best < 0) return OR_DEGENERATE;
    double Eref[9];
    std::memcpy(Eref, bestE, sizeof(Eref));
    or_epi_refine(w, bestE, best_score, Eref, nullptr);
    double U[9], V[9], E2[9];
    or_essential_project(Eref, E2, U, V);
    double R[36], t[12];
    or_essential_candidates(U, V, R, t);
    int cand = 0;
    int64_t cmax = -1;
    for (int i = 0; i < 4; ++i) {
        const int64_t c = or_epi_cheirality(w, R + 9 * i, t + 3 * i);
        if (c > cmax) { cmax = c; cand = i; }
    }
    if (candidate_out) *candidate_out = cand;
    double T1[16] = {0};
    for (int r = 0; r < 3; ++r) {
        for (int c = 0; c < 3; ++c) T1[r * 4 + c] = R[9 * cand + r * 3 + c];
        T1[r * 4 + 3] = baseline * t[3 * cand + r];
    }
    T1[15] = 1.0;
    std::memcpy(T1_out, T1, sizeof(T1));
    or_bootstrap(w, T1);
    return OR_OK;
}


// ---------------------------------------------------------------------------
// Absolute scale from the ground plane (Sec. 6.1: the mode of the pixels whose
// surface normal is near perpendicular; the paper's appendix with the details
// is not part of its text). Readings:
//  - P_j = theta_j K^-1 [x y 1]^T; the normal of pixel j is the unit
//    (P(x+1,y) - P(x-1,y)) x (P(x,y+1) - P(x,y-1)), turned to face the camera
//    (n . P < 0); border pixels, pixels with a neighbour at either end of the
//    depth range, and pixels with mean rigidness over the frames below 1/2 are
//    skipped;
//  - ground candidates: below the camera (P_y > 0, the image y axis pointing
//    down) with |n . (0, 1, 0)| >= cos(max_tilt);
//  - each candidate's camera height is the distance |n . P| of its tangent
//    plane from the camera centre;
//  - the histogram of log2(height) over [-8, 8) in 4096 bins; the bin m of the
//    largest count of the 5-bin box-filtered histogram (the lowest on ties);
//    the mode is the count-weighted mean of the bin centres of the raw
//    histogram over bins m-2 .. m+2;
//  - scale = camera_height / 2^mode (multiply translations and depths by it).
// ---------------------------------------------------------------------------
static void ground_point(const or_window* w, int x, int y, double P[3])
{
    const double th = w->theta[(size_t)y * w->width + x];
    P[0] = th * (x - w->cx) / w->fx;
    P[1] = th * (y - w->cy) / w->fy;
    P[2] = th;
}

int or_ground_scale(const or_window* w, double camera_height, double max_tilt_rad, double* scale_out,
                    double* mode_log2_out, int64_t* candidates_out)
{
    const int W = w->width, H = w->height, T = w->T;
    const int nb = 4096;
    const double lo = -8.0, hi = 8.0, binw = (hi - lo) / nb;
    const double dmin = 1.0 / w->p.inv_depth_max, dmax = 1.0 / w->p.inv_depth_min;
    const double cthr = std::cos(max_tilt_rad);
    std::vector<int64_t> hist(nb, 0);
    int64_t cand = 0;
    for (int y = 1; y < H - 1; ++y) {
        for (int x = 1; x < W - 1; ++x) {
            const size_t j = (size_t)y * W + x;
            bool ok = true;
            const size_t nbj[5] = {j, j - 1, j + 1, j - W, j + W};
            for (int i = 0; i < 5; ++i) {
                const double th = w->theta[nbj[i]];
                if (!(th > dmin && th < dmax)) ok = false;
            }
            double wm = 0.0;
            for (int t = 0; t < T; ++t) wm += w->wmap[(size_t)t * W * H + j];
            if (!ok || !(wm / T >= 0.5)) continue;
            double P[3], Pl[3], Pr[3], Pu[3], Pd[3];
            ground_point(w, x, y, P);
            ground_point(w, x - 1, y, Pl); ground_point(w, x + 1, y, Pr);
            ground_point(w, x, y - 1, Pu); ground_point(w, x, y + 1, Pd);
            double a[3], c[3], n[3];
            sub3(Pr, Pl, a);
            sub3(Pd, Pu, c);
            cross3(a, c, n);
            if (!normalize3(n)) continue;
            if (dot3(n, P) > 0) { n[0] = -n[0]; n[1] = -n[1]; n[2] = -n[2]; }
            if (!(P[1] > 0.0) || !(std::fabs(n[1]) >= cthr)) continue;
            const double h = std::fabs(dot3(n, P));
            if (!(h > 0.0)) continue;
            const double l = std::log2(h);
            if (!(l >= lo && l < hi)) continue;
            int bin = (int)std::floor((l - lo) / binw);
            if (bin >= nb) bin = nb - 1;
            hist[bin] += 1;
            ++cand;
        }
    }
    if (candidates_out) *candidates_out = cand;
    if (cand == 0) return OR_DEGENERATE;
    std::vector<int64_t> sm(nb, 0);
    for (int i = 0; i < nb; ++i)
        for (int k = -2; k <= 2; ++k)
            if (i + k >= 0 && i + k < nb) sm[i] += hist[i + k];
    int m = 0;
    for (int i = 1; i < nb; ++i)
        if (sm[i] > sm[m]) m = i;
    double num = 0.0, cnt = 0.0;
    for (int k = -2; k <= 2; ++k)
        if (m + k >= 0 && m + k < nb) {
            num += (double)hist[m + k] * (lo + (m + k + 0.5) * binw);
            cnt += (double)hist[m + k];
        }
    const double mode = num / cnt;
    if (mode_log2_out) *mode_log2_out = mode;
    if (scale_out) *scale_out = camera_height / std::exp2(mode);
    return OR_OK;
}

}  // extern "C"
