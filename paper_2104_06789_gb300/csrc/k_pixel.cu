// Per-pixel kernels of the VOLDOR loop: bootstrap triangulation, frame pose
// setup, pose preparation (dense-scoring records), E-step emissions and
// forward-backward smoothing, MIE depth sweep, unsmoothed rigidness.
//
// This translation unit is compiled without FMA contraction (--fmad=false):
// the MIE sweep compares a candidate scored in one kernel with one scored in
// another, and equal depths must give bit-identical scores. Fused
// multiply-adds are written out with fmaf where they are wanted.
#include "voldor_internal.cuh"

namespace vd {

// ---------------------------------------------------------------------------
// Frame setup: C_{t-1} = T_{t-1} ... T_1 (FP64) and T_t in the scaled
// cancellation-free form, cast to FP32 for per-pixel work (Eq. 1).
// ---------------------------------------------------------------------------
__global__ void k_frame_setup(DevParams p, DevState s)
{
    const int t = threadIdx.x + 1;
    if (t > p.T) return;
    double C[12] = {1, 0, 0, 0, 0, 1, 0, 0, 0, 0, 1, 0};
    for (int i = 1; i < t; ++i) {
        const double* A = s.poses + 12 * (i - 1);
        double O[12];
        for (int r = 0; r < 3; ++r) {
            for (int c = 0; c < 3; ++c)
                O[r * 4 + c] = A[r * 4 + 0] * C[c] + A[r * 4 + 1] * C[4 + c] + A[r * 4 + 2] * C[8 + c];
            O[r * 4 + 3] = A[r * 4 + 0] * C[3] + A[r * 4 + 1] * C[7] + A[r * 4 + 2] * C[11] + A[r * 4 + 3];
        }
        for (int q = 0; q < 12; ++q) C[q] = O[q];
    }
    for (int q = 0; q < 12; ++q) s.cum[12 * (t - 1) + q] = C[q];
    FrameF f;
    for (int r = 0; r < 3; ++r) {
        for (int c = 0; c < 3; ++c) f.Rc[r * 3 + c] = (float)C[r * 4 + c];
        f.tc[r] = (float)C[r * 4 + 3];
    }
    const double* Tt = s.poses + 12 * (t - 1);
    const double q = p.fyd / p.fxd;
    const double sc[3] = {1.0, q, 1.0};
    for (int r = 0; r < 3; ++r) {
        for (int c = 0; c < 3; ++c) f.E[r * 3 + c] = (float)(sc[r] * (Tt[r * 4 + c] - (r == c ? 1.0 : 0.0)) / sc[c]);
        f.tt[r] = (float)(sc[r] * Tt[r * 4 + 3]);
    }
    s.frames[t - 1] = f;
}

void launch_frame_setup(const DevParams& p, const DevState& s, cudaStream_t st)
{
    k_frame_setup<<<1, 32, 0, st>>>(p, s);
}

// ---------------------------------------------------------------------------
// Bootstrap (Table 1): W := 1, poses := T_1, k := 0, and per pixel the
// least-squares depth along the ray of pixel j from x_j + X_1^j ~ pi_1(theta).
// With d = K^-1 [x y 1], m = K^-1 [x+u y+v 1], R d = d + E d:
//   a_x = (R d)_x - m_x (R d)_z,  b_x = m_x t_z - t_x  (same for y),
//   theta = (a.b)/(a.a), i.e. inverse depth (a.a)/(a.b), clamped.
// ---------------------------------------------------------------------------
struct BootPose {
    double T[12];
    float E[9];
    float t[3];
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
    const float dx = ((float)x - p.cx) * p.inv_fx;
    const float dy = ((float)y - p.cy) * p.inv_fy;
    const float2 f = load_flow(s.flows, p.flow_f16, (size_t)j);
    const float Edx = fmaf(bp.E[0], dx, fmaf(bp.E[1], dy, bp.E[2]));
    const float Edy = fmaf(bp.E[3], dx, fmaf(bp.E[4], dy, bp.E[5]));
    const float Edz = fmaf(bp.E[6], dx, fmaf(bp.E[7], dy, bp.E[8]));
    const float mu_x = f.x * p.inv_fx, mu_y = f.y * p.inv_fy;      // m - d
    const float Rdz = 1.f + Edz;
    const float ax = Edx - dx * Edz - mu_x * Rdz;
    const float ay = Edy - dy * Edz - mu_y * Rdz;
    const float mx = dx + mu_x, my = dy + mu_y;
    const float bx = fmaf(mx, bp.t[2], -bp.t[0]);
    const float by = fmaf(my, bp.t[2], -bp.t[1]);
    const float num = fmaf(ax, ax, ay * ay);
    const float den = fmaf(ax, bx, ay * by);
    float inv = p.inv_depth_min;
    if (den > 0.f) {
        const float r = num / den;
        if (isfinite(r)) inv = fminf(fmaxf(r, p.inv_depth_min), p.inv_depth_max);
    }
    s.theta[j] = 1.f / inv;
}

void launch_bootstrap(const DevParams& p, const DevState& s, const double* T1, cudaStream_t st)
{
    BootPose bp;
    for (int r = 0; r < 3; ++r) {
        for (int c = 0; c < 3; ++c) {
            bp.T[r * 4 + c] = T1[r * 4 + c];
            bp.E[r * 3 + c] = (float)(T1[r * 4 + c] - (r == c ? 1.0 : 0.0));
        }
        bp.T[r * 4 + 3] = T1[r * 4 + 3];
        bp.t[r] = (float)T1[r * 4 + 3];
    }
    const int nb = (p.N + kPixThreads - 1) / kPixThreads;
    k_bootstrap<<<nb, kPixThreads, 0, st>>>(p, s, bp);
}

// ---------------------------------------------------------------------------
// Pose preparation of frame t: one record per pixel whose pi_{t-1} is valid,
// compacted in pixel order (count pass, then write pass with block offsets).
// ---------------------------------------------------------------------------
__global__ void k_prep_count(DevParams p, DevState s, int t)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    __shared__ FrameF fr;
    if (threadIdx.x == 0) fr = s.frames[t - 1];
    __syncthreads();
    bool valid = false;
    if (j < p.N) {
        PixGeom g;
        valid = pixel_geometry(p, fr, s.flows, t, j % p.W, j / p.W, s.theta[j], g);
    }
    const int cnt = __syncthreads_count(valid);
    if (threadIdx.x == 0) s.pix_block_count[blockIdx.x] = cnt;
}

__global__ void k_prep_write(DevParams p, DevState s, int t)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    __shared__ FrameF fr;
    __shared__ int warp_sum[kPixThreads / 32];
    __shared__ int base;
    if (threadIdx.x == 0) fr = s.frames[t - 1];
    // offset of this block: sum of the counts of all earlier blocks
    int acc = 0;
    for (int b = threadIdx.x; b < (int)blockIdx.x; b += blockDim.x) acc += s.pix_block_count[b];
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) warp_sum[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        int tot = 0;
        for (int w = 0; w < kPixThreads / 32; ++w) tot += warp_sum[w];
        base = tot;
    }
    __syncthreads();
    bool valid = false;
    PixGeom g;
    if (j < p.N) valid = pixel_geometry(p, fr, s.flows, t, j % p.W, j / p.W, s.theta[j], g);
    // rank within the block
    const unsigned bal = __ballot_sync(0xffffffffu, valid);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) warp_sum[warp] = __popc(bal);
    __syncthreads();
    int rank = __popc(bal & ((1u << lane) - 1u));
    for (int w = 0; w < warp; ++w) rank += warp_sum[w];
    if (valid) {
        const FiskConst fc = fisk_const(p, g.vob);
        PixRec r;
        r.a = make_float4(g.xb, g.yb2, g.w, g.vob.x * p.inv_fx);
        r.b = make_float4(g.vob.y * p.inv_fx, fc.beta, fc.beta_k, fc.Cp);
        r.c = make_float4(s.wmap[(size_t)(t - 1) * p.N + j], 0.f, 0.f, 0.f);
        s.pix[base + rank] = r;
    }
    if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) {
        int tot = base;
        for (int w = 0; w < kPixThreads / 32; ++w) tot += warp_sum[w];
        *s.pix_count = tot;
    }
}

void launch_pose_prep(const DevParams& p, const DevState& s, int t, cudaStream_t st)
{
    const int nb = (p.N + kPixThreads - 1) / kPixThreads;
    k_prep_count<<<nb, kPixThreads, 0, st>>>(p, s, t);
    k_prep_write<<<nb, kPixThreads, 0, st>>>(p, s, t);
}

// ---------------------------------------------------------------------------
// Per-(t, j) evaluation at a given depth: log[rho/(rho+mu)], log(1/2) where
// the model takes rho := mu.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float frame_ell(const DevParams& p, const FrameF& fr, const void* flows, int t, int x,
                                           int y, float depth)
{
    PixGeom g;
    if (!pixel_geometry(p, fr, flows, t, x, y, depth, g)) return -0.69314718055994531f;
    const FiskConst fc = fisk_const(p, g.vob);
    return pixel_ell(p, fr, g, fc);
}

// Emissions rho/(rho+mu) of every (t, j) at the current depth (E-step input)
// or, written into W, the unsmoothed rigidness update.
__global__ void k_emissions(DevParams p, DevState s, float* out)
{
    __shared__ FrameF frs[kMaxT];
    if (threadIdx.x < p.T) frs[threadIdx.x] = s.frames[threadIdx.x];
    __syncthreads();
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= p.N) return;
    const int x = j % p.W, y = j / p.W;
    const float depth = s.theta[j];
    for (int t = 1; t <= p.T; ++t) {
        const float ell = frame_ell(p, frs[t - 1], s.flows, t, x, y, depth);
        out[(size_t)(t - 1) * p.N + j] = expf(ell);
    }
}

void launch_emissions(const DevParams& p, const DevState& s, float* out, cudaStream_t st)
{
    const int nb = (p.N + kPixThreads - 1) / kPixThreads;
    k_emissions<<<nb, kPixThreads, 0, st>>>(p, s, out);
}

// ---------------------------------------------------------------------------
// Forward-backward (Eqs. 12-14) on every chain of every frame, one thread per
// chain. Emissions (1 - w, w) are read from s.qs and replaced by the
// smoothed q(W = 1). Messages are renormalised at every step; both
// components are kept so that neither loses relative precision.
// ---------------------------------------------------------------------------
__global__ void k_forward_backward(DevParams p, DevState s)
{
    const int dir = (*s.iter) & 3;
    const bool rows = (dir == 0 || dir == 2);
    const int n_chains = rows ? p.H : p.W;
    const int len = rows ? p.W : p.H;
    const int stride = rows ? 1 : p.W;
    const int id = blockIdx.x * blockDim.x + threadIdx.x;
    if (id >= p.T * n_chains) return;
    const int t = id / n_chains, c = id % n_chains;
    const size_t base = (size_t)t * p.N + (rows ? (size_t)c * p.W : (size_t)c);
    float* e = s.qs + base;
    float2* fw = reinterpret_cast<float2*>(s.fb_fwd) + base;
    const float g = p.gamma, h = 1.f - p.gamma;
    float f0, f1;
    {
        const float w = e[0];
        const float a0 = 1.f - w, a1 = w, sum = a0 + a1;
        f0 = a0 / sum;
        f1 = a1 / sum;
        fw[0] = make_float2(f0, f1);
    }
    for (int i = 1; i < len; ++i) {
        const float w = e[(size_t)i * stride];
        const float p0 = g * f0 + h * f1, p1 = h * f0 + g * f1;
        const float a0 = (1.f - w) * p0, a1 = w * p1, sum = a0 + a1;
        f0 = a0 / sum;
        f1 = a1 / sum;
        fw[(size_t)i * stride] = make_float2(f0, f1);
    }
    float b0 = 1.f, b1 = 1.f;
    float w_next = e[(size_t)(len - 1) * stride];
    {
        const float2 f = fw[(size_t)(len - 1) * stride];
        const float q0 = f.x * b0, q1 = f.y * b1;
        e[(size_t)(len - 1) * stride] = q1 / (q0 + q1);
    }
    for (int i = len - 2; i >= 0; --i) {
        const float c0 = (1.f - w_next) * b0, c1 = w_next * b1;
        const float n0 = g * c0 + h * c1, n1 = h * c0 + g * c1, sum = n0 + n1;
        b0 = n0 / sum;
        b1 = n1 / sum;
        w_next = e[(size_t)i * stride];
        const float2 f = fw[(size_t)i * stride];
        const float q0 = f.x * b0, q1 = f.y * b1;
        e[(size_t)i * stride] = q1 / (q0 + q1);
    }
}

void launch_forward_backward(const DevParams& p, const DevState& s, cudaStream_t st)
{
    const int n = p.T * (p.H > p.W ? p.H : p.W);
    k_forward_backward<<<(n + 127) / 128, 128, 0, st>>>(p, s);
}

// ---------------------------------------------------------------------------
// MIE depth update (Eq. 10, Fig. 5).
// Prepare: per pixel, the scores of the prev and smp candidates
// (sum over t of q_s * ell, in order t = 1..T) and the smp depth.
// Sweep: one warp per chain, lane t-1 evaluates frame t of the nbr candidate.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float nan_to_ninf(float v) { return isnan(v) ? -INFINITY : v; }

__global__ void k_mie_prepare(DevParams p, DevState s)
{
    __shared__ FrameF frs[kMaxT];
    if (threadIdx.x < p.T) frs[threadIdx.x] = s.frames[threadIdx.x];
    __syncthreads();
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= p.N) return;
    const int k = *s.iter;
    const int x = j % p.W, y = j / p.W;
    const U64x4 r = philox4x64_10((uint64_t)j, 0ull, (uint64_t)k, (uint64_t)kStreamDepth, p.seed, p.window_id);
    const float u = (float)(r.v[0] >> 40) * (1.f / 16777216.f);
    const float smp = 1.f / fmaf(u, p.inv_depth_max - p.inv_depth_min, p.inv_depth_min);
    const float prev = s.theta[j];
    float sp = 0.f, ss = 0.f;
    for (int t = 1; t <= p.T; ++t) {
        const float q = s.qs[(size_t)(t - 1) * p.N + j];
        sp = __fadd_rn(sp, __fmul_rn(q, frame_ell(p, frs[t - 1], s.flows, t, x, y, prev)));
        ss = __fadd_rn(ss, __fmul_rn(q, frame_ell(p, frs[t - 1], s.flows, t, x, y, smp)));
    }
    s.mie_prev_score[j] = nan_to_ninf(sp);
    s.mie_smp[j] = smp;
    s.mie_smp_score[j] = nan_to_ninf(ss);
}

__global__ void k_mie_sweep(DevParams p, DevState s)
{
    const int dir = (*s.iter) & 3;
    const bool rows = (dir == 0 || dir == 2);
    const int n_chains = rows ? p.H : p.W;
    const int len = rows ? p.W : p.H;
    const int lane = threadIdx.x & 31;
    const int c = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (c >= n_chains) return;
    FrameF fr;
    if (lane < p.T) fr = s.frames[lane];
    const int t = lane + 1;
    float nbr = 0.f;
    for (int i = 0; i < len; ++i) {
        int x, y;
        switch (dir) {
            case 0: x = i; y = c; break;
            case 1: x = c; y = i; break;
            case 2: x = p.W - 1 - i; y = c; break;
            default: x = c; y = p.H - 1 - i; break;
        }
        const int j = y * p.W + x;
        float best = s.theta[j];
        float best_s = s.mie_prev_score[j];
        unsigned char label = 0;
        if (i > 0) {
            float e = 0.f;
            if (lane < p.T) {
                const float q = s.qs[(size_t)(t - 1) * p.N + j];
                e = __fmul_rn(q, frame_ell(p, fr, s.flows, t, x, y, nbr));
            }
            float tot = 0.f;
            for (int tt = 0; tt < p.T; ++tt) tot = __fadd_rn(tot, __shfl_sync(0xffffffffu, e, tt));
            tot = nan_to_ninf(tot);
            if (tot > best_s) { best = nbr; best_s = tot; label = 1; }
        }
        const float ss = s.mie_smp_score[j];
        if (ss > best_s) { best = s.mie_smp[j]; best_s = ss; label = 2; }
        if (lane == 0) {
            s.theta[j] = best;
            s.labels[j] = label;
        }
        nbr = best;
    }
}

void launch_mie(const DevParams& p, const DevState& s, cudaStream_t st)
{
    const int nb = (p.N + kPixThreads - 1) / kPixThreads;
    k_mie_prepare<<<nb, kPixThreads, 0, st>>>(p, s);
    const int chains = p.H > p.W ? p.H : p.W;
    const int warps_per_block = 4;
    k_mie_sweep<<<(chains + warps_per_block - 1) / warps_per_block, 32 * warps_per_block, 0, st>>>(p, s);
}

// ---------------------------------------------------------------------------
// Iteration counter.
// ---------------------------------------------------------------------------
__global__ void k_set_iter(int* iter, int k) { *iter = k; }
__global__ void k_advance_iter(int* iter) { *iter += 1; }

void launch_set_iteration(const DevState& s, int k, cudaStream_t st) { k_set_iter<<<1, 1, 0, st>>>(s.iter, k); }
void launch_advance_iteration(const DevState& s, cudaStream_t st) { k_advance_iter<<<1, 1, 0, st>>>(s.iter); }

}  // namespace vd
