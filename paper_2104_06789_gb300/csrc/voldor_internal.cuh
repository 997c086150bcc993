// Internal declarations of the sm_103a VOLDOR library: device parameter block,
// context layout, device helpers shared by the kernels, and the host-side
// launchers each translation unit provides.
#pragma once

#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <stdint.h>
#include <stddef.h>

#include "voldor.h"

namespace vd {

constexpr int kMaxT = 16;
constexpr int kMaxSols = 4;            // P3P has at most four solutions
constexpr int kScoreThreads = 256;     // dense scoring block
constexpr int kScoreHypsPerThread = 8;   // hypotheses per thread of the allocation-free scoring (ILP)
constexpr int kScoreDefaultHpt = 2;      // a window's dense-scoring shape until autotuned: 2 hypotheses
constexpr int kScoreDefaultWaves = 8;    // per thread, three blocks per SM, pixel chunks for 8 waves
constexpr int kScoreBlocksPerSM = 1;
constexpr int kScoreHypsPerBlock = kScoreThreads * kScoreHypsPerThread;
constexpr int kMeanshiftCtas = 8;      // thread-block cluster of the meanshift
constexpr int kMeanshiftThreads = 256;
constexpr int kPixThreads = 256;
constexpr int kScoreLogMax = 1024;
// Status word 3 of a window: a count of frames whose pose update was
// degenerate, plus this bit when a bounded device-side wait gave up.
constexpr int kStatusTimeout = 1 << 30;
constexpr int kTuneMaxWaves = 8;       // largest dense-scoring grid the autotuner tries, in waves
constexpr int kMaxImageSide = 4096;   // longest chain the depth sweep resolves in shared memory

// Everything a kernel needs to know about the window, by value.
struct DevParams {
    int W, H, T, N;
    int S, G, ms_max_iter, flow_f16;
    int criterion;                      // VOLDOR_CRITERION_MIE or _MLE
    int residual;                       // VOLDOR_RESIDUAL_FISK or _GAUSSIAN
    float fx, fy, cx, cy, inv_fx, inv_fy, fy_over_fx;
    float log2_a1, a2_log2e, b1, b2, beta_min, lambda2;
    float x_min, x_max;                 // px^2
    float xs_min, xs_max;               // scaled by 1/fx^2
    float log2_fx2;
    float inv_depth_min, inv_depth_max;
    float gamma;
    double fxd, fyd, cxd, cyd;
    double inv_fxd, inv_fyd, fy_over_fx_d;
    double sigma_t, sigma_r, ms_tol;
    uint64_t seed, window_id;
    // fx, fy, cx, cy, 1/fx, 1/fy as float-float pairs (hi, lo) for the df32
    // geometry passes
    float kdf[12];
    unsigned w_magic;                   // floor(2^32 / W): pixel index -> row without a division
};

// (x, y) of pixel j: q = hi32(j floor(2^32 / W)) is floor(j / W) or one less,
// and one comparison corrects it (exact for 0 <= j < 2^31).
__device__ __forceinline__ void pixel_xy(const DevParams& p, int j, int& x, int& y)
{
    unsigned q = __umulhi((unsigned)j, p.w_magic);
    unsigned r = (unsigned)j - q * (unsigned)p.W;
    if (r >= (unsigned)p.W) { ++q; r -= (unsigned)p.W; }
    x = (int)r;
    y = (int)q;
}

// Per-pixel record of a frame for dense scoring (three float4 = 48 B).
//  a = {xb, yb2, w, ut}: normalised coords x/z, (fy/fx) y/z, inverse depth 1/z
//      in camera t-1, observed flow u / fx
//  b = {vt, beta, beta_k, Cp}: observed flow v / fx, Fisk shape, beta *
//      log2(fx^2 / alpha), mu / beta * fx^2; under the Gaussian residual
//      model {vt, fx^2 / alpha, -x_mu / alpha, 0}
//  c = {wq, 0, 0, 0}: rigidness weight W_t^j
struct PixRec {
    float4 a, b, c;
};

// Device state of a window (all pointers are device memory).
struct DevState {
    const void* flows;        // [T][H][W] float2 or __half2
    float* theta;             // [H][W]
    float* wmap;              // [T][H][W] unsmoothed W
    float* qs;                // [T][H][W] smoothed q (also emission scratch)
    double* poses;            // [T][12] row-major [R | t]
    double* cum;              // [T][12] C_{t-1} = T_{t-1} ... T_1 (FP64)
    float* frames32;          // [T][24] FP32 E_c = R_c - I, t_c, E_t = R_t - I, t_t
    float* cum_df;            // [T][12][2] C_{t-1} as float-float pairs (hi, lo)
    float* poses_df;          // [T][12][2] T_t as float-float pairs
    int* iter;                // [1] iteration counter k
    int* status;              // [4] n_hyp, seed, meanshift steps, status bits
    // dense scoring scratch
    PixRec* pix;              // [N] compacted valid pixels of the current frame
    int* pix_block_count;     // [ceil(N / kPixThreads)] valid pixels per block, then the blocks' record offsets
    unsigned* prep_done;      // [1] blocks of the count pass finished (0 between launches)
    int* pix_count;           // [1]
    unsigned* pix_vmask;      // [ceil(N / kPixThreads) * kPixThreads / 32] per-warp ballots of the valid pixels
    // P3P
    int* p3p_claims;          // [1] 32-group chunks claimed by the P3P warps of the current frame
    unsigned long long* p3p_done;   // [1] chunks solved (high 32 bits) and their solutions (low 32 bits)
    double* grp_sols;         // [G][4][12]
    double* grp_weight;       // [G]
    int* grp_count;           // [G]
    int* grp_offset;          // [G]
    int* n_hyp;               // [1]
    double* hyp_Rt;           // [S][12]
    float* hyp_f32;           // [S][12] scoring form
    float* hyp_pw;            // [S][16] se(3) log as float-float (hi of the 6 coordinates, then lo), group weight, 0 0 0
    double* hyp_w;            // [S]
    float* hyp_dp;            // [S][8] meanshift scratch: p_h - p_seed (6), w_h, 0
    long long* hyp_info;      // [S][2]
    double* partial;          // [n_chunks][S]
    double* scores;           // [S]
    // depth sweep
    float* mie_prev_score;    // [N]
    float* mie_smp;           // [N]
    float* mie_smp_score;     // [N]
    int* mie_next;            // [N] end of each pixel's speculative run (chain position), negative if capped
    unsigned char* labels;    // [N]
    float* fb_fwd;            // [T][H][W] forward messages
    long long* score_log;     // [kScoreLogMax][2] (n_hyp, n_pix) of timed scoring launches
    int n_chunks;             // dense scoring pixel chunks
    int score_hpt;            // dense scoring hypotheses per thread (2, 4 or 8)
};

// ---------------------------------------------------------------------------
// Philox4x64-10 (Salmon, Moraes, Dror, Shaw, SC'11).
// ---------------------------------------------------------------------------
struct U64x4 { uint64_t v[4]; };

__device__ __forceinline__ U64x4 philox4x64_10(uint64_t c0, uint64_t c1, uint64_t c2, uint64_t c3,
                                                uint64_t k0, uint64_t k1)
{
    const uint64_t mA = 0xD2E7470EE14C6C93ULL, mB = 0xCA5A826395121157ULL;
    const uint64_t wA = 0x9E3779B97F4A7C15ULL, wB = 0xBB67AE8584CAA73BULL;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint64_t hiA = __umul64hi(mA, c0), loA = mA * c0;
        const uint64_t hiB = __umul64hi(mB, c2), loB = mB * c2;
        const uint64_t n0 = hiB ^ c1 ^ k0;
        const uint64_t n2 = hiA ^ c3 ^ k1;
        c0 = n0; c1 = loB; c2 = n2; c3 = loA;
        k0 += wA; k1 += wB;
    }
    U64x4 o;
    o.v[0] = c0; o.v[1] = c1; o.v[2] = c2; o.v[3] = c3;
    return o;
}

enum { kStreamPose = 1, kStreamDepth = 2, kStreamEpi = 3 };

// ---------------------------------------------------------------------------
// Flow access.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float2 load_flow(const void* flows, int flow_f16, size_t idx)
{
    if (flow_f16) {
        const __half2 h = reinterpret_cast<const __half2*>(flows)[idx];
        return __half22float2(h);
    }
    return reinterpret_cast<const float2*>(flows)[idx];
}

// Bilinear lookup of frame t (0-based ft) at (u, v); false outside
// [0, W-1] x [0, H-1].
__device__ __forceinline__ bool flow_bilinear(const DevParams& p, const void* flows, int ft, float u, float v,
                                              float2& out)
{
    if (!(u >= 0.f && u <= (float)(p.W - 1) && v >= 0.f && v <= (float)(p.H - 1))) return false;
    int x0 = min((int)floorf(u), p.W - 2);
    int y0 = min((int)floorf(v), p.H - 2);
    const float ax = u - (float)x0, ay = v - (float)y0;
    const size_t base = (size_t)ft * p.N + (size_t)y0 * p.W + x0;
    const float2 f00 = load_flow(flows, p.flow_f16, base);
    const float2 f10 = load_flow(flows, p.flow_f16, base + 1);
    const float2 f01 = load_flow(flows, p.flow_f16, base + p.W);
    const float2 f11 = load_flow(flows, p.flow_f16, base + p.W + 1);
    const float w00 = (1.f - ax) * (1.f - ay), w10 = ax * (1.f - ay), w01 = (1.f - ax) * ay, w11 = ax * ay;
    out.x = w00 * f00.x + w10 * f10.x + w01 * f01.x + w11 * f11.x;
    out.y = w00 * f00.y + w10 * f10.y + w01 * f01.y + w11 * f11.y;
    return true;
}

// ---------------------------------------------------------------------------
// Per-pixel geometry (Eq. 1) is FP64 in the per-pixel passes because the rigid
// flow (tens of px) cancels against the observed flow down to residuals of a
// tenth of a pixel; the likelihood arithmetic that follows is FP32.
// ---------------------------------------------------------------------------

// 1/d in FP64 from the SFU reciprocal and two Newton steps (full double
// precision for normal d; falls back to division outside [1e-30, 1e30]).
__device__ __forceinline__ double rcp64(double d)
{
    const double ad = fabs(d);
    if (!(ad > 1e-30 && ad < 1e30)) return 1.0 / d;
    double r = (double)__frcp_rn((float)d);
    double e = fma(-d, r, 1.0);
    r = fma(r, e, r);
    e = fma(-d, r, 1.0);
    return fma(r, e, r);
}

// Stages C_{t-1} and T_t of every frame in shared memory.
struct FramesD {
    double C[kMaxT][12];
    double Tt[kMaxT][12];
};

__device__ __forceinline__ void load_frames(const DevParams& p, const DevState& s, FramesD& f)
{
    for (int i = threadIdx.x; i < p.T * 12; i += blockDim.x) {
        f.C[i / 12][i % 12] = s.cum[i];
        f.Tt[i / 12][i % 12] = s.poses[i];
    }
    __syncthreads();
}

// Fisk quantities of an observed flow of magnitude n (Eqs. 5-7), FP32:
// beta, log2(alpha), and mu / beta written as ys / (x_mu (1 + ys)^2) with
// x_mu = lambda^2 n^2 and ys = 2^-|beta log2(x_mu / alpha)|.
struct FiskConst {
    float beta, log2_alpha, mu_over_beta;
};

__device__ __forceinline__ FiskConst fisk_const(const DevParams& p, float n)
{
    FiskConst c;
    c.log2_alpha = fmaf(p.a2_log2e, n, p.log2_a1);
    c.beta = fmaxf(fmaf(p.b1, n, p.b2), p.beta_min);
    const float xmu = fminf(fmaxf(p.lambda2 * n * n, p.x_min), p.x_max);
    const float smu = c.beta * (log2f(xmu) - c.log2_alpha);
    const float ys = exp2f(-fabsf(smu));
    const float g = 1.f + ys;
    c.mu_over_beta = ys / (xmu * g * g);
    return c;
}

// Gaussian residual model (the ablation study's alternative, Sec. 6.3): the
// squared EPE x is exponential with the Fisk median alpha(n) (reading:
// variance matched by the median), so log2(mu / rho) = (x - x_mu) / alpha.
struct GaussConst {
    float inv_alpha, x_mu;
};

__device__ __forceinline__ GaussConst gauss_const(const DevParams& p, float n)
{
    GaussConst c;
    c.inv_alpha = exp2f(-fmaf(p.a2_log2e, n, p.log2_a1));
    c.x_mu = fminf(fmaxf(p.lambda2 * n * n, p.x_min), p.x_max);
    return c;
}

// -(the criterion's term) of one (t, j) in FP32 from the clamped squared
// residual x (px^2) and the observed flow magnitude n: log(1 + mu/rho)
// (MIE, Eq. 10) or log(mu/rho) (MLE, Eq. 9), under the window's residual model.
//   Fisk:     mu / rho = (mu / beta) x (y + 2 + 1/y),  y = (x / alpha)^beta
//   Gaussian: mu / rho = 2^s,  s = (x - x_mu) / alpha; log(1 + 2^s) taken as
//             max(s, 0) ln 2 + log1p(2^-|s|) (finite for any s)
__device__ __forceinline__ float neg_ell(const DevParams& p, float x, float n, bool mle)
{
    if (p.residual == VOLDOR_RESIDUAL_GAUSSIAN) {
        const GaussConst gc = gauss_const(p, n);
        const float s = (x - gc.x_mu) * gc.inv_alpha;
        return mle ? s * 0.69314718055994531f : fmaxf(s, 0.f) * 0.69314718055994531f + log1pf(exp2f(-fabsf(s)));
    }
    const FiskConst fc = fisk_const(p, n);
    const float s = fc.beta * (log2f(x) - fc.log2_alpha);
    const float e = exp2f(fabsf(s));
    const float r = fc.mu_over_beta * x * (e + 2.f + 1.f / e);
    return mle ? logf(r) : log1pf(r);
}

// ---------------------------------------------------------------------------
// Host-side launchers (one translation unit each).
// ---------------------------------------------------------------------------
void launch_frame_setup(const DevParams& p, const DevState& s, cudaStream_t st);
void launch_bootstrap(const DevParams& p, const DevState& s, const double* T1, cudaStream_t st);
void launch_pose_prep(const DevParams& p, const DevState& s, int t, cudaStream_t st);
void launch_prep_count(const DevParams& p, const DevState& s, int t, cudaStream_t st);
void launch_prep_write(const DevParams& p, const DevState& s, int t, cudaStream_t st);
void launch_p3p_groups(const DevParams& p, const DevState& s, int t, cudaStream_t st);
void launch_hyp_collect(const DevParams& p, const DevState& s, cudaStream_t st);
void launch_hyp_log(const DevParams& p, const DevState& s, cudaStream_t st);
void launch_score(const DevParams& p, const DevState& s, int log_idx, cudaStream_t st);
void launch_score_reduce(const DevParams& p, const DevState& s, cudaStream_t st);
void launch_meanshift(const DevParams& p, const DevState& s, int t, cudaStream_t st);
void launch_emissions(const DevParams& p, const DevState& s, float* out, cudaStream_t st);
void launch_forward_backward(const DevParams& p, const DevState& s, cudaStream_t st);
void launch_mie(const DevParams& p, const DevState& s, cudaStream_t st);
void launch_set_iteration(const DevState& s, int k, cudaStream_t st);
void launch_advance_iteration(const DevState& s, cudaStream_t st);
int score_chunks(int S, int N);
// Learned proposal over a triangulated bootstrap state (flags: VOLDOR_LEARNED_*);
// *kernels gets the number of kernels launched.
voldor_status net_bootstrap(voldor_net* n, const void* flows, int f16, int W, int H, int T, float d_min, float d_max, int flags,
                            float* theta, float* wmap, cudaStream_t st, int* kernels);
// Epipolar bootstrap scratch (a separate allocation of the context, sized by
// the number of samples M; the correspondence records reuse the pose
// preparation's pixel-record buffer).
struct EpiState {
    int M;                    // samples
    float4* rec;              // [N] calibrated correspondences (NaN: invalid)
    int* valid;               // [M] 1 valid; -1 repeated pixel, -2 target outside I_1, -3 rank < 8, -4 rank(E) < 2
    double* E;                // [M][9] projected essential matrix
    double* UV;               // [M][18] U, V (row-major, det +1)
    float* form;              // [M][12] Q = R - I (9), t (3)
    unsigned* hist;           // [3][M][kEpiBins]
    unsigned* prefix;         // [M] bits selected so far
    unsigned* rank;           // [M] remaining rank
    float* median;            // [M]
    long long* info;          // [8]: chosen, candidate, n_valid, n_inliers, count[4]
    double* partial;          // [blocks][46] A^T A partials (45) + inlier count
    double* refined;          // [9 E][9 U][9 V]
    double* cand;             // [4][12] [R | t]
    double* T1;               // [12]
    int partial_blocks;
};
size_t epi_scratch_bytes(int M);
size_t epi_layout(void* base, int M, float4* rec, EpiState* e);
int launch_epipolar(const DevParams& p, const DevState& s, const EpiState& e, double baseline, cudaStream_t st);
// Ground-plane scale: hist [4096] and out [3] are device scratch; returns the
// number of kernels launched.
constexpr int kGroundScratchBytes = 4096 * 4 + 256;
int launch_ground_scale(const DevParams& p, const DevState& s, double camera_height, double cos_tilt, double dmin,
                        double dmax, int apply, unsigned* hist, double* out, cudaStream_t st);
int score_chunks_for(int S, int N, int hpt, int waves);
int score_chunks_max(int S, int N);
void score_hyps_from_host(const DevParams& p, const DevState& s, int n, cudaStream_t st);

}  // namespace vd
