// FP64-geometry passes of the VOLDOR loop: pose preparation (the dense
// scoring's per-pixel records), the E-step emissions (also the unsmoothed
// rigidness update) and forward-backward smoothing of the rigidness.
//
// Geometry is FP64 and likelihood arithmetic FP32 (k_prep_count/k_prep_write,
// k_emissions, neg_ell). Unlike the MIE sweep's translation unit this one is
// compiled with FMA contraction: none of its results is compared bit for bit
// with another kernel's, and fused FP64 multiply-adds cut the FP64
// instructions of the geometry (this GPU's FP64 rate is a small fraction of
// its FP32 rate).
#include "voldor_internal.cuh"

namespace vd {

// ---------------------------------------------------------------------------
// Pose preparation of frame t: one record per pixel whose pi_{t-1} is valid,
// compacted in pixel order. The count pass computes each pixel's point in
// camera t-1, P = C_{t-1} theta K^-1 [x y 1] (FP64), its reciprocal depth and
// pi_{t-1}, stores them (SoA, pix_geo[6][N]) and counts the valid pixels per
// block, and its last block to finish scans the counts into block offsets;
// the write pass reads them back (valid iff P_z > 0 and pi_{t-1} inside the
// image, the same test on the same values), samples the flow at pi_{t-1}
// bilinearly (FP64) and writes the records at its block's offset.
// ---------------------------------------------------------------------------
__global__ void k_prep_count(DevParams p, DevState s, int t)
{
    __shared__ double C[12];
    if (threadIdx.x < 12) C[threadIdx.x] = s.cum[12 * (t - 1) + threadIdx.x];
    __syncthreads();
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    bool valid = false;
    if (j < p.N) {
        const int x = j % p.W, y = j / p.W;
        const double th = (double)s.theta[j];
        const double dx = ((double)x - p.cxd) * p.inv_fxd, dy = ((double)y - p.cyd) * p.inv_fyd;
        double Px = th * dx, Py = th * dy, Pz = th, u = (double)x, v = (double)y, iz = 0.0;
        if (t > 1) {
            const double X = Px, Y = Py, Z = Pz;
            Px = C[0] * X + C[1] * Y + C[2] * Z + C[3];
            Py = C[4] * X + C[5] * Y + C[6] * Z + C[7];
            Pz = C[8] * X + C[9] * Y + C[10] * Z + C[11];
        }
        if (Pz > 0.0) {
            iz = rcp64(Pz);
            if (t > 1) {
                u = p.fxd * Px * iz + p.cxd;
                v = p.fyd * Py * iz + p.cyd;
            }
        }
        valid = Pz > 0.0 && u >= 0.0 && u <= (double)(p.W - 1) && v >= 0.0 && v <= (double)(p.H - 1);
        const size_t N = (size_t)p.N;
        s.pix_geo[j] = Px;
        s.pix_geo[N + j] = Py;
        s.pix_geo[2 * N + j] = Pz;
        s.pix_geo[3 * N + j] = u;
        s.pix_geo[4 * N + j] = v;
        s.pix_geo[5 * N + j] = iz;
    }
    // per-warp ballots of the valid pixels: with the block offsets they map
    // the i-th valid pixel (pixel order) to its index for the minimal groups
    const unsigned bal = __ballot_sync(0xffffffffu, valid);
    if ((threadIdx.x & 31) == 0) s.pix_vmask[j >> 5] = bal;
    const int cnt = __syncthreads_count(valid);
    // the last block to finish turns the block counts into block offsets
    // (exclusive scan, in place), sets the record count and clears the P3P
    // claim counters of the frame; no block waits
    __shared__ bool last;
    if (threadIdx.x == 0) {
        s.pix_block_count[blockIdx.x] = cnt;
        __threadfence();
        last = atomicAdd(s.prep_done, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    const int nb = gridDim.x, per = (nb + blockDim.x - 1) / blockDim.x;
    const int b0 = min((int)threadIdx.x * per, nb), b1 = min(b0 + per, nb);
    volatile int* counts = s.pix_block_count;
    int local = 0;
    for (int b = b0; b < b1; ++b) local += counts[b];
    __shared__ int wsum[kPixThreads / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int incl = local;
    for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += v;
    }
    if (lane == 31) wsum[warp] = incl;
    __syncthreads();
    int before = 0;
    for (int w = 0; w < warp; ++w) before += wsum[w];
    int off = before + incl - local;
    for (int b = b0; b < b1; ++b) {
        const int c = counts[b];
        counts[b] = off;
        off += c;
    }
    if (threadIdx.x == blockDim.x - 1) {
        *s.pix_count = off;
        *s.prep_done = 0u;
        *s.p3p_claims = 0;
        *s.p3p_done = 0ull;
    }
}

__global__ void k_prep_write(DevParams p, DevState s, int t)
{
    __shared__ int warp_sum[kPixThreads / 32];
    const int base = s.pix_block_count[blockIdx.x];      // this block's offset (set by the count pass)
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    const size_t N = (size_t)p.N;
    bool valid = false;
    double Px = 0.0, Py = 0.0, iz = 0.0, u = 0.0, v = 0.0;
    if (j < p.N) {
        Px = s.pix_geo[j];
        Py = s.pix_geo[N + j];
        const double Pz = s.pix_geo[2 * N + j];
        u = s.pix_geo[3 * N + j];
        v = s.pix_geo[4 * N + j];
        iz = s.pix_geo[5 * N + j];
        valid = Pz > 0.0 && u >= 0.0 && u <= (double)(p.W - 1) && v >= 0.0 && v <= (double)(p.H - 1);
    }
    const unsigned bal = __ballot_sync(0xffffffffu, valid);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) warp_sum[warp] = __popc(bal);
    __syncthreads();
    int rank = __popc(bal & ((1u << lane) - 1u));
    for (int w = 0; w < warp; ++w) rank += warp_sum[w];
    if (valid) {
        const int x0 = min((int)floor(u), p.W - 2), y0 = min((int)floor(v), p.H - 2);
        const double ax = u - x0, ay = v - y0;
        const size_t fb = (size_t)(t - 1) * N + (size_t)y0 * p.W + x0;
        const float2 f00 = load_flow(s.flows, p.flow_f16, fb), f10 = load_flow(s.flows, p.flow_f16, fb + 1);
        const float2 f01 = load_flow(s.flows, p.flow_f16, fb + p.W);
        const float2 f11 = load_flow(s.flows, p.flow_f16, fb + p.W + 1);
        const double w00 = (1.0 - ax) * (1.0 - ay), w10 = ax * (1.0 - ay), w01 = (1.0 - ax) * ay, w11 = ax * ay;
        const double fu = w00 * f00.x + w10 * f10.x + w01 * f01.x + w11 * f11.x;
        const double fv = w00 * f00.y + w10 * f10.y + w01 * f01.y + w11 * f11.y;
        const float n = sqrtf((float)(fu * fu + fv * fv));
        PixRec r;
        r.a = make_float4((float)(Px * iz), (float)(p.fy_over_fx_d * Py * iz), (float)iz, (float)(fu * p.inv_fxd));
        if (p.residual == VOLDOR_RESIDUAL_GAUSSIAN) {
            const GaussConst gc = gauss_const(p, n);
            r.b = make_float4((float)(fv * p.inv_fxd), (float)(p.fxd * p.fxd) * gc.inv_alpha, -gc.x_mu * gc.inv_alpha,
                              0.f);
        } else {
            const FiskConst fc = fisk_const(p, n);
            r.b = make_float4((float)(fv * p.inv_fxd), fc.beta, fc.beta * (p.log2_fx2 - fc.log2_alpha),
                              (float)(p.fxd * p.fxd) * fc.mu_over_beta);
        }
        r.c = make_float4(s.wmap[(size_t)(t - 1) * N + j], 0.f, 0.f, 0.f);
        s.pix[base + rank] = r;
    }
}

void launch_prep_count(const DevParams& p, const DevState& s, int t, cudaStream_t st)
{
    const int nb = (p.N + kPixThreads - 1) / kPixThreads;
    k_prep_count<<<nb, kPixThreads, 0, st>>>(p, s, t);
}

void launch_prep_write(const DevParams& p, const DevState& s, int t, cudaStream_t st)
{
    const int nb = (p.N + kPixThreads - 1) / kPixThreads;
    k_prep_write<<<nb, kPixThreads, 0, st>>>(p, s, t);
}

void launch_pose_prep(const DevParams& p, const DevState& s, int t, cudaStream_t st)
{
    launch_prep_count(p, s, t, st);
    launch_prep_write(p, s, t, st);
}

// Emissions rho/(rho+mu) of every (t, j) at the current depth (E-step input)
// or, written into W, the unsmoothed rigidness update: per (t, j) the rigid
// flow and residual in FP64 and the likelihood in FP32 (neg_ell); log(1/2)
// where the model takes rho := mu (pi_{t-1} invalid or the point behind camera
// t). The point is carried from frame to frame: the point in camera
// t (T_t applied to the point in camera t-1) and its projection pi_t are the
// next frame's point in camera (t+1)-1 and pi_{(t+1)-1}, since C_t X =
// T_t (C_{t-1} X), so each frame transforms and projects once (FP64).
__global__ void k_emissions(DevParams p, DevState s, float* out)
{
    __shared__ FramesD f;
    load_frames(p, s, f);
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= p.N) return;
    const int x = j % p.W, y = j / p.W;
    const double th = (double)s.theta[j];
    const double dx = ((double)x - p.cxd) * p.inv_fxd, dy = ((double)y - p.cyd) * p.inv_fyd;
    double Px = th * dx, Py = th * dy, Pz = th;     // the point in camera t-1 (camera 0 for t = 1)
    double u = (double)x, v = (double)y;            // pi_{t-1}
    bool front = th > 0.0;                          // P_z > 0 and (u, v) defined
    for (int t = 1; t <= p.T; ++t) {
        float ell = -0.69314718055994531f;          // rho := mu
        double fu = 0.0, fv = 0.0;
        const bool valid_prev =
            front && u >= 0.0 && u <= (double)(p.W - 1) && v >= 0.0 && v <= (double)(p.H - 1);
        if (valid_prev) {
            const int x0 = min((int)floor(u), p.W - 2), y0 = min((int)floor(v), p.H - 2);
            const double ax = u - x0, ay = v - y0;
            const size_t base = (size_t)(t - 1) * p.N + (size_t)y0 * p.W + x0;
            const float2 f00 = load_flow(s.flows, p.flow_f16, base), f10 = load_flow(s.flows, p.flow_f16, base + 1);
            const float2 f01 = load_flow(s.flows, p.flow_f16, base + p.W);
            const float2 f11 = load_flow(s.flows, p.flow_f16, base + p.W + 1);
            const double w00 = (1.0 - ax) * (1.0 - ay), w10 = ax * (1.0 - ay), w01 = (1.0 - ax) * ay, w11 = ax * ay;
            fu = w00 * f00.x + w10 * f10.x + w01 * f01.x + w11 * f11.x;
            fv = w00 * f00.y + w10 * f10.y + w01 * f01.y + w11 * f11.y;
        }
        const double* Tt = f.Tt[t - 1];
        const double Qx = Tt[0] * Px + Tt[1] * Py + Tt[2] * Pz + Tt[3];
        const double Qy = Tt[4] * Px + Tt[5] * Py + Tt[6] * Pz + Tt[7];
        const double Qz = Tt[8] * Px + Tt[9] * Py + Tt[10] * Pz + Tt[11];
        const bool front_t = Qz > 0.0;
        double uq = 0.0, vq = 0.0;
        if (front_t) {
            const double iq = rcp64(Qz);
            uq = p.fxd * Qx * iq + p.cxd;
            vq = p.fyd * Qy * iq + p.cyd;
        }
        if (valid_prev && front_t) {
            const double ru = (uq - u) - fu, rv = (vq - v) - fv;
            const float xs = (float)fmin(fmax(ru * ru + rv * rv, (double)p.x_min), (double)p.x_max);
            ell = -neg_ell(p, xs, sqrtf((float)(fu * fu + fv * fv)), false);
        }
        out[(size_t)(t - 1) * p.N + j] = expf(ell);
        Px = Qx; Py = Qy; Pz = Qz;
        u = uq; v = vq;
        front = front_t;
    }
}

void launch_emissions(const DevParams& p, const DevState& s, float* out, cudaStream_t st)
{
    const int nb = (p.N + kPixThreads - 1) / kPixThreads;
    k_emissions<<<nb, kPixThreads, 0, st>>>(p, s, out);
}

// ---------------------------------------------------------------------------
// Forward-backward (Eqs. 12-14) on every chain of every frame, one warp per
// chain. Emissions (1 - w, w) are read from s.qs and replaced by the
// smoothed q(W = 1). With A = [[g, h], [h, g]] (g = gamma, h = 1 - gamma):
//   forward   f_0 = e_0,  f_i = diag(e_i) A f_{i-1}
//   backward  b_{n-1} = 1, b_i = A diag(e_{i+1}) b_{i+1}
//   q_i = f_i .* b_i (normalised),
// every message renormalised at every step. The chain is cut into 32
// contiguous segments, one per lane; each lane forms the product of its
// segment's 2x2 transfer matrices (renormalised by their entry sum, all
// entries are non-negative), a 5-step shuffle scan gives each lane the
// product of the segments before it (forward) or after it (backward), and
// each lane then walks its own segment with the step-by-step recursion from
// the message entering it.
// ---------------------------------------------------------------------------
struct M22 {
    float a, b, c, d;   // [[a, b], [c, d]]
};

__device__ __forceinline__ M22 m22_mul(const M22& x, const M22& y)
{
    M22 r{x.a * y.a + x.b * y.c, x.a * y.b + x.b * y.d, x.c * y.a + x.d * y.c, x.c * y.b + x.d * y.d};
    const float s = r.a + r.b + r.c + r.d;
    if (s > 0.f) {
        const float is = 1.f / s;
        r.a *= is; r.b *= is; r.c *= is; r.d *= is;
    }
    return r;
}

__device__ __forceinline__ M22 m22_shfl(const M22& x, int src_delta, bool up)
{
    M22 r;
    if (up) {
        r.a = __shfl_up_sync(0xffffffffu, x.a, src_delta); r.b = __shfl_up_sync(0xffffffffu, x.b, src_delta);
        r.c = __shfl_up_sync(0xffffffffu, x.c, src_delta); r.d = __shfl_up_sync(0xffffffffu, x.d, src_delta);
    } else {
        r.a = __shfl_down_sync(0xffffffffu, x.a, src_delta); r.b = __shfl_down_sync(0xffffffffu, x.b, src_delta);
        r.c = __shfl_down_sync(0xffffffffu, x.c, src_delta); r.d = __shfl_down_sync(0xffffffffu, x.d, src_delta);
    }
    return r;
}

__global__ void __launch_bounds__(256) k_forward_backward(DevParams p, DevState s)
{
    const int dir = (*s.iter) & 3;
    const bool rows = (dir == 0 || dir == 2);
    const int n_chains = rows ? p.H : p.W;
    const int len = rows ? p.W : p.H;
    const int stride = rows ? 1 : p.W;
    const int lane = threadIdx.x & 31;
    const int id = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (id >= p.T * n_chains) return;                // whole warps leave together
    const int t = id / n_chains, c = id % n_chains;
    const size_t base = (size_t)t * p.N + (rows ? (size_t)c * p.W : (size_t)c);
    float* e = s.qs + base;
    float2* fw = reinterpret_cast<float2*>(s.fb_fwd) + base;
    const float g = p.gamma, h = 1.f - p.gamma;
    const int L = (len + 31) / 32;
    const int i0 = min(lane * L, len), i1 = min(i0 + L, len);    // this lane's segment [i0, i1)
    const bool has = i0 < i1;

    // ---- forward: segment products of diag(e_i) A for i in [max(i0, 1), i1)
    M22 P{1.f, 0.f, 0.f, 1.f};
    for (int i = (i0 > 0 ? i0 : 1); i < i1; ++i) {
        const float w = e[(size_t)i * stride];
        const M22 Mi{(1.f - w) * g, (1.f - w) * h, w * h, w * g};
        P = m22_mul(Mi, P);
    }
    // inclusive scan: S_k = P_k ... P_0 (later segments on the left)
    M22 S = P;
    for (int d = 1; d < 32; d <<= 1) {
        const M22 o = m22_shfl(S, d, true);
        if (lane >= d) S = m22_mul(S, o);
    }
    const M22 Sprev = m22_shfl(S, 1, true);          // S_{k-1}
    float f0, f1;
    {
        const float w = e[0];
        const float a0 = 1.f - w, a1 = w, sum = a0 + a1;
        f0 = a0 / sum;
        f1 = a1 / sum;
    }
    if (lane > 0) {                                   // f_{i0 - 1} = S_{k-1} f_0
        const float a0 = Sprev.a * f0 + Sprev.b * f1, a1 = Sprev.c * f0 + Sprev.d * f1, sum = a0 + a1;
        f0 = a0 / sum;
        f1 = a1 / sum;
    }
    if (has) {
        int i = i0;
        if (i == 0) {
            fw[0] = make_float2(f0, f1);
            i = 1;
        }
        for (; i < i1; ++i) {
            const float w = e[(size_t)i * stride];
            const float p0 = g * f0 + h * f1, p1 = h * f0 + g * f1;
            const float a0 = (1.f - w) * p0, a1 = w * p1, sum = a0 + a1;
            f0 = a0 / sum;
            f1 = a1 / sum;
            fw[(size_t)i * stride] = make_float2(f0, f1);
        }
    }

    // ---- backward: segment products of A diag(e_{i+1}) for i in [i0, min(i1, len - 1))
    const int j1 = min(i1, len - 1);
    M22 R{1.f, 0.f, 0.f, 1.f};
    for (int i = j1 - 1; i >= i0; --i) {
        const float w = e[(size_t)(i + 1) * stride];
        const M22 Ni{g * (1.f - w), h * w, h * (1.f - w), g * w};
        R = m22_mul(Ni, R);                           // N_i ... N_{j1 - 1}
    }
    // the emission just past this segment, read before any lane writes q
    const float w_after = i1 < len ? e[(size_t)i1 * stride] : 0.f;
    // suffix scan: U_k = R_k R_{k+1} ... R_31
    M22 U = R;
    for (int d = 1; d < 32; d <<= 1) {
        const M22 o = m22_shfl(U, d, false);
        if (lane + d < 32) U = m22_mul(U, o);
    }
    const M22 Unext = m22_shfl(U, 1, false);          // U_{k+1}
    float b0 = 1.f, b1 = 1.f;                          // b_{len - 1}
    if (lane < 31 && i1 < len) {                       // b_{i1} = U_{k+1} 1
        const float n0 = Unext.a + Unext.b, n1 = Unext.c + Unext.d, sum = n0 + n1;
        b0 = n0 / sum;
        b1 = n1 / sum;
    }
    __syncwarp();                                      // every lane has read its emissions
    if (has) {
        float w_next = w_after;
        int i = i1 - 1;
        if (i1 == len) {                               // the chain's last element: b = 1
            w_next = e[(size_t)i * stride];
            const float2 f = fw[(size_t)i * stride];
            const float q0 = f.x * b0, q1 = f.y * b1;
            e[(size_t)i * stride] = q1 / (q0 + q1);
            --i;
        }
        for (; i >= i0; --i) {
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
}

void launch_forward_backward(const DevParams& p, const DevState& s, cudaStream_t st)
{
    const int n = p.T * (p.H > p.W ? p.H : p.W);      // chains (warps) of the longer count
    k_forward_backward<<<(n + 7) / 8, 256, 0, st>>>(p, s);
}

}  // namespace vd
