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
#include "df32.cuh"
#include "voldor_internal.cuh"

namespace vd {

// ---------------------------------------------------------------------------
// Pose preparation of frame t: one record per pixel whose pi_{t-1} is valid,
// compacted in pixel order. Both passes compute each pixel's point in camera
// t-1, P = C_{t-1} theta K^-1 [x y 1], and pi_{t-1} in df32 (float-float on
// the FP32 pipe, ~44 bits: the validity test 0 <= pi_{t-1} <= size - 1 and
// the bilinear sample position are those of an FP64 computation but within
// ~1e-11 px). The count pass counts the valid pixels per block and stores
// per-warp ballots of them, and its last block to finish scans the counts
// into block offsets; the write pass recomputes the same values, samples the
// flow at pi_{t-1} bilinearly (df32) and writes the records at its block's
// offset.
// ---------------------------------------------------------------------------
struct PrepGeo {
    DF Px, Py, Pz, u, v;
    bool valid;
};

// C_{t-1} as float-float pairs, written by the frame set-up
__device__ __forceinline__ void load_cum_df(const DevState& s, int t, DF* C)
{
    if (threadIdx.x < 12) {
        const float* c = s.cum_df + 24 * (t - 1) + 2 * threadIdx.x;
        C[threadIdx.x] = DF{c[0], c[1]};
    }
    __syncthreads();
}

__device__ __forceinline__ PrepGeo prep_geometry(const DevParams& p, const DF* C, int t, int j, float th)
{
    int x, y;
    pixel_xy(p, j, x, y);
    const DF fx{p.kdf[0], p.kdf[1]}, fy{p.kdf[2], p.kdf[3]}, cx{p.kdf[4], p.kdf[5]}, cy{p.kdf[6], p.kdf[7]};
    const DF ifx{p.kdf[8], p.kdf[9]}, ify{p.kdf[10], p.kdf[11]};
    PrepGeo g;
    const float xf = small_int_to_float(x), yf = small_int_to_float(y);
    const DF X = df_mul(df_mul(df_add(df_neg(cx), xf), ifx), th);
    const DF Y = df_mul(df_mul(df_add(df_neg(cy), yf), ify), th);
    const DF Z = df_of(th);
    g.u = df_of(xf);
    g.v = df_of(yf);
    if (t == 1) {
        g.Px = X; g.Py = Y; g.Pz = Z;
    } else {
        g.Px = df_add(df_add(df_mul(C[0], X), df_mul(C[1], Y)), df_add(df_mul(C[2], Z), C[3]));
        g.Py = df_add(df_add(df_mul(C[4], X), df_mul(C[5], Y)), df_add(df_mul(C[6], Z), C[7]));
        g.Pz = df_add(df_add(df_mul(C[8], X), df_mul(C[9], Y)), df_add(df_mul(C[10], Z), C[11]));
    }
    g.valid = df_gt0(g.Pz);
    if (g.valid && t > 1) {
        const DF iz = df_div(df_of(1.f), g.Pz);
        g.u = df_add(df_mul(df_mul(fx, g.Px), iz), cx);
        g.v = df_add(df_mul(df_mul(fy, g.Py), iz), cy);
    }
    g.valid = g.valid && df_ge(g.u, 0.f) && df_le(g.u, small_int_to_float(p.W - 1)) && df_ge(g.v, 0.f) &&
              df_le(g.v, small_int_to_float(p.H - 1));
    return g;
}

__global__ void __launch_bounds__(kPixThreads) k_prep_count(DevParams p, DevState s, int t)
{
    __shared__ DF C[12];
    load_cum_df(s, t, C);
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    bool valid = false;
    if (j < p.N) valid = prep_geometry(p, C, t, j, s.theta[j]).valid;
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

__global__ void __launch_bounds__(kPixThreads) k_prep_write(DevParams p, DevState s, int t)
{
    __shared__ DF C[12];
    __shared__ int warp_sum[kPixThreads / 32];
    load_cum_df(s, t, C);
    const int base = s.pix_block_count[blockIdx.x];      // this block's offset (set by the count pass)
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    const size_t N = (size_t)p.N;
    PrepGeo g;
    g.valid = false;
    if (j < p.N) g = prep_geometry(p, C, t, j, s.theta[j]);
    const unsigned bal = __ballot_sync(0xffffffffu, g.valid);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) warp_sum[warp] = __popc(bal);
    __syncthreads();
    int rank = __popc(bal & ((1u << lane) - 1u));
    for (int w = 0; w < warp; ++w) rank += warp_sum[w];
    if (g.valid) {
        const int x0 = min(df_floor(g.u), p.W - 2), y0 = min(df_floor(g.v), p.H - 2);
        const DF ax = df_add(g.u, -small_int_to_float(x0)), ay = df_add(g.v, -small_int_to_float(y0));
        const size_t fb = (size_t)(t - 1) * N + (size_t)y0 * p.W + x0;
        const float2 f00 = load_flow(s.flows, p.flow_f16, fb), f10 = load_flow(s.flows, p.flow_f16, fb + 1);
        const float2 f01 = load_flow(s.flows, p.flow_f16, fb + p.W);
        const float2 f11 = load_flow(s.flows, p.flow_f16, fb + p.W + 1);
        const DF gu0 = df_add(df_mul(df_two_sum(f10.x, -f00.x), ax), f00.x);
        const DF gu1 = df_add(df_mul(df_two_sum(f11.x, -f01.x), ax), f01.x);
        const DF gv0 = df_add(df_mul(df_two_sum(f10.y, -f00.y), ax), f00.y);
        const DF gv1 = df_add(df_mul(df_two_sum(f11.y, -f01.y), ax), f01.y);
        const DF fud = df_add(gu0, df_mul(df_sub(gu1, gu0), ay));
        const DF fvd = df_add(gv0, df_mul(df_sub(gv1, gv0), ay));
        const DF ifx{p.kdf[8], p.kdf[9]};
        const float fu = df_to_float(fud), fv = df_to_float(fvd);
        const float ut = df_to_float(df_mul(fud, ifx)), vt = df_to_float(df_mul(fvd, ifx));
        const DF iz = df_div(df_of(1.f), g.Pz);
        const float n = sqrtf(fmaf(fu, fu, fv * fv));
        const float fx2 = df_to_float(df_mul(DF{p.kdf[0], p.kdf[1]}, DF{p.kdf[0], p.kdf[1]}));
        PixRec r;
        r.a = make_float4(df_to_float(df_mul(g.Px, iz)), df_to_float(df_mul(df_mul(g.Py, iz), p.fy_over_fx)),
                          df_to_float(iz), ut);
        if (p.residual == VOLDOR_RESIDUAL_GAUSSIAN) {
            const GaussConst gc = gauss_const(p, n);
            r.b = make_float4(vt, fx2 * gc.inv_alpha, -gc.x_mu * gc.inv_alpha, 0.f);
        } else {
            const FiskConst fc = fisk_const(p, n);
            r.b = make_float4(vt, fc.beta, fc.beta * (p.log2_fx2 - fc.log2_alpha), fx2 * fc.mu_over_beta);
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
// flow and residual in df32 (float-float, on the FP32 pipe) and the
// likelihood in FP32 (neg_ell); log(1/2) where the model takes rho := mu
// (pi_{t-1} invalid or the point behind camera t). The point is carried from
// frame to frame: the point in camera t (T_t applied to the point in camera
// t-1) and its projection pi_t are the next frame's point in camera (t+1)-1
// and pi_{(t+1)-1}, since C_t X = T_t (C_{t-1} X), so each frame transforms
// and projects once (the frame set-up's float-float copy of T_t). The residual xi - v_ob (tenths of a pixel) is the
// difference of quantities of up to hundreds of pixels: the sample position,
// the bilinear flow (in lerp form, with df32 fractions) and the rigid flow
// are all kept in df32 and only the residual is rounded to FP32.
__global__ void __launch_bounds__(kPixThreads) k_emissions(DevParams p, DevState s, float* out)
{
    __shared__ DF Tdf[kMaxT][12];
    for (int i = threadIdx.x; i < p.T * 12; i += blockDim.x)
        Tdf[i / 12][i % 12] = DF{s.poses_df[2 * i], s.poses_df[2 * i + 1]};
    __syncthreads();
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= p.N) return;
    int x, y;
    pixel_xy(p, j, x, y);
    const DF fx{p.kdf[0], p.kdf[1]}, fy{p.kdf[2], p.kdf[3]}, cx{p.kdf[4], p.kdf[5]}, cy{p.kdf[6], p.kdf[7]};
    const DF ifx{p.kdf[8], p.kdf[9]}, ify{p.kdf[10], p.kdf[11]};
    const float th = s.theta[j];
    // the point in camera t-1 (camera 0 for t = 1) and pi_{t-1}
    const float xf = small_int_to_float(x), yf = small_int_to_float(y);
    DF Px = df_mul(df_mul(df_add(df_neg(cx), xf), ifx), th);
    DF Py = df_mul(df_mul(df_add(df_neg(cy), yf), ify), th);
    DF Pz = df_of(th);
    DF u = df_of(xf), v = df_of(yf);
    bool front = th > 0.f;                          // P_z > 0 and (u, v) defined
    const float Wm1 = small_int_to_float(p.W - 1), Hm1 = small_int_to_float(p.H - 1);
    for (int t = 1; t <= p.T; ++t) {
        float ell = -0.69314718055994531f;          // rho := mu
        DF fu = df_of(0.f), fv = df_of(0.f);
        const bool valid_prev = front && df_ge(u, 0.f) && df_le(u, Wm1) && df_ge(v, 0.f) && df_le(v, Hm1);
        if (valid_prev) {
            const int x0 = min(df_floor(u), p.W - 2), y0 = min(df_floor(v), p.H - 2);
            const DF ax = df_add(u, -small_int_to_float(x0)), ay = df_add(v, -small_int_to_float(y0));
            const size_t base = (size_t)(t - 1) * p.N + (size_t)y0 * p.W + x0;
            const float2 f00 = load_flow(s.flows, p.flow_f16, base), f10 = load_flow(s.flows, p.flow_f16, base + 1);
            const float2 f01 = load_flow(s.flows, p.flow_f16, base + p.W);
            const float2 f11 = load_flow(s.flows, p.flow_f16, base + p.W + 1);
            // f00 + ax (f10 - f00), f01 + ax (f11 - f01), then the same in y
            const DF gu0 = df_add(df_mul(df_two_sum(f10.x, -f00.x), ax), f00.x);
            const DF gu1 = df_add(df_mul(df_two_sum(f11.x, -f01.x), ax), f01.x);
            const DF gv0 = df_add(df_mul(df_two_sum(f10.y, -f00.y), ax), f00.y);
            const DF gv1 = df_add(df_mul(df_two_sum(f11.y, -f01.y), ax), f01.y);
            fu = df_add(gu0, df_mul(df_sub(gu1, gu0), ay));
            fv = df_add(gv0, df_mul(df_sub(gv1, gv0), ay));
        }
        const DF* Tt = Tdf[t - 1];
        const DF Qx = df_add(df_add(df_mul(Tt[0], Px), df_mul(Tt[1], Py)), df_add(df_mul(Tt[2], Pz), Tt[3]));
        const DF Qy = df_add(df_add(df_mul(Tt[4], Px), df_mul(Tt[5], Py)), df_add(df_mul(Tt[6], Pz), Tt[7]));
        const DF Qz = df_add(df_add(df_mul(Tt[8], Px), df_mul(Tt[9], Py)), df_add(df_mul(Tt[10], Pz), Tt[11]));
        const bool front_t = df_gt0(Qz);
        DF uq = df_of(0.f), vq = df_of(0.f);
        if (front_t) {
            const DF iq = df_div(df_of(1.f), Qz);
            uq = df_add(df_mul(df_mul(fx, Qx), iq), cx);
            vq = df_add(df_mul(df_mul(fy, Qy), iq), cy);
        }
        if (valid_prev && front_t) {
            const float ru = df_to_float(df_sub(df_sub(uq, u), fu));
            const float rv = df_to_float(df_sub(df_sub(vq, v), fv));
            const float xs = fminf(fmaxf(fmaf(ru, ru, rv * rv), p.x_min), p.x_max);
            const float fuf = df_to_float(fu), fvf = df_to_float(fv);
            ell = -neg_ell(p, xs, sqrtf(fmaf(fuf, fuf, fvf * fvf)), false);
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
