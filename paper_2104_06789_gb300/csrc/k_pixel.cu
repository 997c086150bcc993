// Per-pixel kernels of the VOLDOR loop: frame pose setup, bootstrap
// triangulation and the MIE depth sweep (the FP64-geometry passes are in
// k_geom.cu).
//
// This translation unit is compiled without FMA contraction (--fmad=false):
// the MIE sweep compares a candidate scored in one kernel with one scored in
// another, and equal depths must give bit-identical scores.
#include "voldor_internal.cuh"

namespace vd {

// ---------------------------------------------------------------------------
// Frame setup: C_{t-1} = T_{t-1} ... T_1 for every t (FP64), the product of
// Eq. 1 with T_t the motion from t-1 to t.
// ---------------------------------------------------------------------------
// One warp: the poses are staged in shared memory, then thread c < 4 carries
// column c of C (O = A C is column by column: O[:, c] = A[:, :3] C[:, c], plus
// A's translation for c = 3), each element added in the same order as the
// row-by-row product.
__global__ void k_frame_setup(DevParams p, DevState s)
{
    __shared__ double A[kMaxT * 12];
    __shared__ double Cs[kMaxT * 12];          // C_{t-1}, [t - 1][3][4]
    for (int i = threadIdx.x; i < p.T * 12; i += blockDim.x) A[i] = s.poses[i];
    __syncthreads();
    // the product chain C_t = T_t C_{t-1}: thread c < 4 carries column c
    const int c = threadIdx.x;
    if (c < 4) {
        double C0 = c == 0 ? 1.0 : 0.0, C1 = c == 1 ? 1.0 : 0.0, C2 = c == 2 ? 1.0 : 0.0;
        for (int t = 1; t <= p.T; ++t) {
            double* Ct = Cs + 12 * (t - 1);
            Ct[c] = C0;
            Ct[4 + c] = C1;
            Ct[8 + c] = C2;
            const double* At = A + 12 * (t - 1);
            double n0 = At[0] * C0 + At[1] * C1 + At[2] * C2;
            double n1 = At[4] * C0 + At[5] * C1 + At[6] * C2;
            double n2 = At[8] * C0 + At[9] * C1 + At[10] * C2;
            if (c == 3) {
                n0 = n0 + At[3];
                n1 = n1 + At[7];
                n2 = n2 + At[11];
            }
            C0 = n0;
            C1 = n1;
            C2 = n2;
        }
    }
    __syncthreads();
    // every stage's outputs, one element (t, r, col) per thread: C_{t-1} in FP64
    // and as float-float pairs (hi = fl32(v), lo = fl32(v - hi)), T_t as
    // float-float pairs, and both as E = R - I, t in FP32
    for (int i = threadIdx.x; i < p.T * 12; i += blockDim.x) {
        const int t1 = i / 12, e = i % 12, r = e / 4, col = e % 4;
        const double cv = Cs[i], av = A[i];
        s.cum[i] = cv;
        const float ch = (float)cv, ah = (float)av;
        s.cum_df[2 * i] = ch;
        s.cum_df[2 * i + 1] = (float)(cv - (double)ch);
        s.poses_df[2 * i] = ah;
        s.poses_df[2 * i + 1] = (float)(av - (double)ah);
        float* f = s.frames32 + 24 * t1;        // E_c = R_c - I, t_c, E_t = R_t - I, t_t
        if (col < 3) {
            f[3 * r + col] = (float)(cv - (r == col ? 1.0 : 0.0));
            f[12 + 3 * r + col] = (float)(av - (r == col ? 1.0 : 0.0));
        } else {
            f[9 + r] = (float)cv;
            f[21 + r] = (float)av;
        }
    }
}

void launch_frame_setup(const DevParams& p, const DevState& s, cudaStream_t st)
{
    k_frame_setup<<<1, kMaxT * 12, 0, st>>>(p, s);
}

// ---------------------------------------------------------------------------
// Bootstrap (Table 1): W := 1, poses := T_1, k := 0, and per pixel the
// least-squares depth along the ray of pixel j from x_j + X_1^j ~ pi_1(theta).
// With d = K^-1 [x y 1], m = K^-1 [x+u y+v 1]:
//   a_x = (R d)_x - m_x (R d)_z,  b_x = m_x t_z - t_x  (same for y),
//   theta = (a.b)/(a.a), i.e. inverse depth (a.a)/(a.b), clamped; FP64.
// ---------------------------------------------------------------------------
struct BootPose {
    double T[12];
};

__global__ void k_bootstrap(DevParams p, DevState s, BootPose bp)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j == 0) {
        for (int t = 0; t < p.T; ++t)
            for (int q = 0; q < 12; ++q) s.poses[12 * t + q] = bp.T[q];
        *s.iter = 0;
    }
    if (j >= p.N) return;
    for (int t = 0; t < p.T; ++t) s.wmap[(size_t)t * p.N + j] = 1.f;
    const int x = j % p.W, y = j / p.W;
    const double* M = bp.T;
    const double dx = ((double)x - p.cxd) * p.inv_fxd, dy = ((double)y - p.cyd) * p.inv_fyd;
    const float2 f = load_flow(s.flows, p.flow_f16, (size_t)j);
    const double mx = ((double)x + f.x - p.cxd) * p.inv_fxd, my = ((double)y + f.y - p.cyd) * p.inv_fyd;
    const double Rdx = M[0] * dx + M[1] * dy + M[2];
    const double Rdy = M[4] * dx + M[5] * dy + M[6];
    const double Rdz = M[8] * dx + M[9] * dy + M[10];
    const double ax = Rdx - mx * Rdz, bx = mx * M[11] - M[3];
    const double ay = Rdy - my * Rdz, by = my * M[11] - M[7];
    const double num = ax * ax + ay * ay, den = ax * bx + ay * by;
    double inv = (double)p.inv_depth_min;
    if (den > 0.0) {
        const double r = num / den;
        if (isfinite(r)) inv = fmin(fmax(r, (double)p.inv_depth_min), (double)p.inv_depth_max);
    }
    s.theta[j] = (float)(1.0 / inv);
}

void launch_bootstrap(const DevParams& p, const DevState& s, const double* T1, cudaStream_t st)
{
    BootPose bp;
    for (int q = 0; q < 12; ++q) bp.T[q] = T1[q];
    const int nb = (p.N + kPixThreads - 1) / kPixThreads;
    k_bootstrap<<<nb, kPixThreads, 0, st>>>(p, s, bp);
}


// ell_t(j) at depth d in FP32 for the MIE candidate scores, written without
// cancellation: with d = K^-1 [x y 1], the point in camera t-1 is
// theta (d + a), a = E_c d + t_c / theta, so pi_{t-1} = (x, y) + delta with
// delta = f (a_xy - d_xy a_z) / (1 + a_z) (a small quantity); the sample
// position is split into an integer pixel and a fraction; the rigid flow is
// xi = f (b_xy - pb_xy b_z) / (1 + b_z) with b = E_t pb + t_t / P_z. Every
// MIE candidate is scored by this one function, so equal depths score
// bit-identically.
struct FramesF {
    float v[kMaxT][24];
};

__device__ __forceinline__ void load_frames32(const DevParams& p, const DevState& s, FramesF& f)
{
    for (int i = threadIdx.x; i < p.T * 24; i += blockDim.x) f.v[i / 24][i % 24] = s.frames32[i];
    __syncthreads();
}

__device__ __forceinline__ float depth_ell_fast(const DevParams& p, const float* fr, const void* flows, int t, int x,
                                                int y, float depth)
{
    // invalid (t, j): rho := mu, i.e. log 1/2 under MIE and 0 under MLE
    const float ln_half = p.criterion == VOLDOR_CRITERION_MLE ? 0.f : -0.69314718055994531f;
    if (!(depth > 0.f)) return ln_half;
    const float dx = ((float)x - p.cx) * p.inv_fx, dy = ((float)y - p.cy) * p.inv_fy;
    const float w0 = 1.f / depth;
    float pbx = dx, pby = dy, w = w0;
    int x0 = x, y0 = y;
    float fxr = 0.f, fyr = 0.f;
    if (t > 1) {
        const float* E = fr;
        const float ax = fmaf(E[0], dx, fmaf(E[1], dy, fmaf(fr[9], w0, E[2])));
        const float ay = fmaf(E[3], dx, fmaf(E[4], dy, fmaf(fr[10], w0, E[5])));
        const float az = fmaf(E[6], dx, fmaf(E[7], dy, fmaf(fr[11], w0, E[8])));
        const float den = 1.f + az;
        if (!(den > 0.f)) return ln_half;
        const float rd = 1.f / den;
        const float mx = fmaf(-dx, az, ax) * rd, my = fmaf(-dy, az, ay) * rd;    // pb - d
        pbx = dx + mx;
        pby = dy + my;
        w = w0 * rd;
        const float du = p.fx * mx, dv = p.fy * my;     // pi_{t-1} - (x, y)
        if (!(fabsf(du) < 1e7f && fabsf(dv) < 1e7f)) return ln_half;
        const float iu = floorf(du), iv = floorf(dv);
        x0 = x + (int)iu;
        y0 = y + (int)iv;
        fxr = du - iu;
        fyr = dv - iv;
    }
    // valid iff 0 <= u <= W-1 and 0 <= v <= H-1
    if (x0 < 0 || y0 < 0 || x0 > p.W - 1 || y0 > p.H - 1) return ln_half;
    if ((x0 == p.W - 1 && fxr > 0.f) || (y0 == p.H - 1 && fyr > 0.f)) return ln_half;
    if (x0 == p.W - 1) { x0 = p.W - 2; fxr = 1.f; }
    if (y0 == p.H - 1) { y0 = p.H - 2; fyr = 1.f; }
    const size_t base = (size_t)(t - 1) * p.N + (size_t)y0 * p.W + x0;
    const float2 f00 = load_flow(flows, p.flow_f16, base), f10 = load_flow(flows, p.flow_f16, base + 1);
    const float2 f01 = load_flow(flows, p.flow_f16, base + p.W), f11 = load_flow(flows, p.flow_f16, base + p.W + 1);
    const float w00 = (1.f - fxr) * (1.f - fyr), w10 = fxr * (1.f - fyr), w01 = (1.f - fxr) * fyr, w11 = fxr * fyr;
    const float fu = fmaf(w00, f00.x, fmaf(w10, f10.x, fmaf(w01, f01.x, w11 * f11.x)));
    const float fv = fmaf(w00, f00.y, fmaf(w10, f10.y, fmaf(w01, f01.y, w11 * f11.y)));
    const float* Et = fr + 12;
    const float bx = fmaf(Et[0], pbx, fmaf(Et[1], pby, fmaf(fr[21], w, Et[2])));
    const float by = fmaf(Et[3], pbx, fmaf(Et[4], pby, fmaf(fr[22], w, Et[5])));
    const float bz = fmaf(Et[6], pbx, fmaf(Et[7], pby, fmaf(fr[23], w, Et[8])));
    const float den = 1.f + bz;
    if (!(den > 0.f)) return ln_half;
    const float rd = 1.f / den;
    const float ru = fmaf(p.fx * fmaf(-pbx, bz, bx), rd, -fu);
    const float rv = fmaf(p.fy * fmaf(-pby, bz, by), rd, -fv);
    const float xsq = fminf(fmaxf(fmaf(ru, ru, rv * rv), p.x_min), p.x_max);
    // MIE (Eq. 10): log rho/(rho+mu); MLE (Eq. 9): log rho - log mu
    return -neg_ell(p, xsq, sqrtf(fmaf(fu, fu, fv * fv)), p.criterion == VOLDOR_CRITERION_MLE);
}


// ---------------------------------------------------------------------------
// MIE depth update (Eq. 10, Fig. 5), chain-parallel with the exact sequential
// semantics. Along a chain, the sequential sweep carries one value v (the
// winner at the previous pixel) and at position i picks
//   v           if S_i(v) > S_i(prev_i) and S_i(v) >= S_i(smp_i),
//   own_i       otherwise, own_i = smp_i if S_i(smp_i) > S_i(prev_i) else prev_i,
// where S_i(d) = sum_t q_s(t, i) ell_t(i; d) summed in order t = 1..T. So the
// carried value is always own_r of the last position r where it was reset,
// and it survives from r until the first position where it loses. Three
// phases reproduce that bit for bit:
//   prepare  per pixel: S(prev), smp, S(smp), own;
//   runs     per pixel r (in parallel): test own_r at r+1, r+2, ... until it
//            loses, at most kRunCap positions (speculation);
//   resolve  per chain: follow r -> end of run from the chain start; a run
//            that reached the cap is continued on the fly.
// ---------------------------------------------------------------------------
constexpr int kRunCap = 8;

__device__ __forceinline__ float nan_to_ninf(float v) { return isnan(v) ? -INFINITY : v; }

__device__ __forceinline__ float mie_score(const DevParams& p, const DevState& s, const FramesF& f, int x, int y, float d)
{
    const int j = y * p.W + x;
    float acc = 0.f;
    for (int t = 1; t <= p.T; ++t) {
        const float q = s.qs[(size_t)(t - 1) * p.N + j];
        acc = __fadd_rn(acc, __fmul_rn(q, depth_ell_fast(p, f.v[t - 1], s.flows, t, x, y, d)));
    }
    return nan_to_ninf(acc);
}

// Chain geometry: (x, y) of position i of chain c in direction dir.
__device__ __forceinline__ void chain_xy(const DevParams& p, int dir, int c, int i, int& x, int& y)
{
    switch (dir) {
        case 0: x = i; y = c; break;
        case 1: x = c; y = i; break;
        case 2: x = p.W - 1 - i; y = c; break;
        default: x = c; y = p.H - 1 - i; break;
    }
}

__device__ __forceinline__ bool survives(const DevState& s, int j, float sv)
{
    return sv > s.mie_prev_score[j] && sv >= s.mie_smp_score[j];
}

__global__ void k_mie_prepare(DevParams p, DevState s)
{
    __shared__ FramesF f;
    load_frames32(p, s, f);
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= p.N) return;
    const int k = *s.iter;
    const int x = j % p.W, y = j / p.W;
    const U64x4 r = philox4x64_10((uint64_t)j, 0ull, (uint64_t)k, (uint64_t)kStreamDepth, p.seed, p.window_id);
    const float u = (float)(r.v[0] >> 40) * (1.f / 16777216.f);
    const float smp = 1.f / fmaf(u, p.inv_depth_max - p.inv_depth_min, p.inv_depth_min);
    s.mie_prev_score[j] = mie_score(p, s, f, x, y, s.theta[j]);
    s.mie_smp[j] = smp;
    s.mie_smp_score[j] = mie_score(p, s, f, x, y, smp);
}

// own value of pixel j (before the sweep overwrites theta)
__device__ __forceinline__ float own_value(const DevState& s, int j)
{
    return s.mie_smp_score[j] > s.mie_prev_score[j] ? s.mie_smp[j] : s.theta[j];
}

__global__ void k_mie_runs(DevParams p, DevState s)
{
    __shared__ FramesF f;
    load_frames32(p, s, f);
    const int dir = (*s.iter) & 3;
    const bool rows = (dir == 0 || dir == 2);
    const int len = rows ? p.W : p.H;
    const int id = blockIdx.x * blockDim.x + threadIdx.x;
    if (id >= p.N) return;
    const int c = id / len, i = id % len;
    int x, y;
    chain_xy(p, dir, c, i, x, y);
    const int j = y * p.W + x;
    const float v = own_value(s, j);
    int e = i + 1;
    int steps = 0;
    while (e < len && steps < kRunCap) {
        int xe, ye;
        chain_xy(p, dir, c, e, xe, ye);
        if (!survives(s, ye * p.W + xe, mie_score(p, s, f, xe, ye, v))) break;
        ++e;
        ++steps;
    }
    s.mie_next[j] = (steps == kRunCap && e < len) ? -e : e;
}

constexpr int kResolveThreads = 128;
constexpr int kMaxChain = kMaxImageSide;

// Resolution of one chain per block. All threads walk the run ends in
// lockstep from the chain start (uniform control flow); a run whose
// speculation reached the cap is continued kResolveThreads positions at a
// time, each thread testing one position; the run's positions are filled in
// parallel.
__global__ void __launch_bounds__(kResolveThreads) k_mie_resolve(DevParams p, DevState s)
{
    __shared__ FramesF f;
    __shared__ short origin[kMaxChain];
    __shared__ int next_s[kMaxChain];
    __shared__ int first_fail;
    load_frames32(p, s, f);
    const int dir = (*s.iter) & 3;
    const bool rows = (dir == 0 || dir == 2);
    const int n_chains = rows ? p.H : p.W;
    const int len = rows ? p.W : p.H;
    const int c = blockIdx.x;
    if (c >= n_chains) return;
    for (int q = threadIdx.x; q < len; q += kResolveThreads) {
        int x, y;
        chain_xy(p, dir, c, q, x, y);
        next_s[q] = s.mie_next[y * p.W + x];
    }
    __syncthreads();
    int r = 0;
    while (r < len) {
        int e = next_s[r];
        if (e < 0) {                           // speculation capped: continue block-parallel
            int xr, yr;
            chain_xy(p, dir, c, r, xr, yr);
            const float v = own_value(s, yr * p.W + xr);
            int pos = -e;
            while (true) {
                if (threadIdx.x == 0) first_fail = len;
                __syncthreads();
                const int q = pos + (int)threadIdx.x;
                if (q < len) {
                    int xe, ye;
                    chain_xy(p, dir, c, q, xe, ye);
                    if (!survives(s, ye * p.W + xe, mie_score(p, s, f, xe, ye, v))) atomicMin(&first_fail, q);
                }
                __syncthreads();
                const int ff = first_fail;
                __syncthreads();
                if (ff < len || pos + kResolveThreads >= len) { e = ff < len ? ff : len; break; }
                pos += kResolveThreads;
            }
        }
        for (int q = r + (int)threadIdx.x; q < e; q += kResolveThreads) origin[q] = (short)r;
        r = e;
    }
    __syncthreads();
    // new depths and labels; read every own value before any theta is written
    float vals[kMaxChain / kResolveThreads];
    unsigned char labs[kMaxChain / kResolveThreads];
    int n = 0;
    for (int q = threadIdx.x; q < len; q += kResolveThreads, ++n) {
        int x, y;
        chain_xy(p, dir, c, origin[q], x, y);
        const int jo = y * p.W + x;
        vals[n] = own_value(s, jo);
        labs[n] = (origin[q] != q) ? 1 : (s.mie_smp_score[jo] > s.mie_prev_score[jo] ? 2 : 0);
    }
    __syncthreads();
    n = 0;
    for (int q = threadIdx.x; q < len; q += kResolveThreads, ++n) {
        int x, y;
        chain_xy(p, dir, c, q, x, y);
        const int j = y * p.W + x;
        s.theta[j] = vals[n];
        s.labels[j] = labs[n];
    }
}

void launch_mie(const DevParams& p, const DevState& s, cudaStream_t st)
{
    const int nb = (p.N + kPixThreads - 1) / kPixThreads;
    k_mie_prepare<<<nb, kPixThreads, 0, st>>>(p, s);
    k_mie_runs<<<nb, kPixThreads, 0, st>>>(p, s);
    k_mie_resolve<<<p.H > p.W ? p.H : p.W, kResolveThreads, 0, st>>>(p, s);
}

// ---------------------------------------------------------------------------
// Iteration counter.
// ---------------------------------------------------------------------------
__global__ void k_set_iter(int* iter, int k) { *iter = k; }
__global__ void k_advance_iter(int* iter) { *iter += 1; }

void launch_set_iteration(const DevState& s, int k, cudaStream_t st) { k_set_iter<<<1, 1, 0, st>>>(s.iter, k); }
void launch_advance_iteration(const DevState& s, cudaStream_t st) { k_advance_iter<<<1, 1, 0, st>>>(s.iter); }

}  // namespace vd
