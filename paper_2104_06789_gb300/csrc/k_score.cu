// Dense hypothesis scoring: for every P3P hypothesis h of frame t,
//   L_h = sum_j W_t^j log[rho_j(h) / (rho_j(h) + mu_j)]
// over the pixels whose pi_{t-1} is valid -- the MIE criterion of Eq. 10 with
// the pose as the free variable (Eq. 9's MLE form as the ablation variant).
//
// Per pair, with the pixel record (xb, yb2, w, ut, vt, beta, beta_k, Cp, wq)
// and the hypothesis in scaled form (E, tt):
//   a    = E (xb, yb2, 1) + tt w                (camera-t point / z_{t-1} - p)
//   r_u  = (a_x - xb a_z) / (1 + a_z) - ut      (residual / fx, no cancellation
//   r_v  = (a_y - yb2 a_z) / (1 + a_z) - vt      against the pixel position)
//   xs   = r_u^2 + r_v^2, clamped to [xs_min, xs_max]  (squared residual / fx^2)
//   s    = beta log2(xs) + beta_k               (log2 of (x/alpha)^beta)
//   r    = Cp xs (2^s + 2 + 2^-s)               (= mu / rho, Eqs. 3-4, 7)
//   ell  = -log1p(r); behind camera t (1 + a_z <= 0) rho := mu, ell = -log 2.
// SFU work: rcp, lg2, ex2, ex2, lg2 (for r >= 1/8); log1p(r) for r < 1/8 is a
// polynomial on the FMA pipe, because lg2 near 1 has only absolute accuracy.
//
// The FP32 add / mul / fma work runs on packed pairs: two hypotheses share a
// 64-bit register pair and one .f32x2 instruction does both lanes, which
// halves the issue slots of the FMA-pipe work (the pipe still does 128 lane
// operations per SM clock: after the SFU it is this kernel's second limit).
// Each thread carries 1 pair (2 hypotheses, three 256-thread blocks per SM:
// the default shape), 2 pairs (4 hypotheses, two blocks per SM) or 4 pairs
// (8 hypotheses, one block per SM); the pixel
// loop is software-pipelined over two consecutive pixels; pixel records are
// bulk-copied into shared memory tile by tile and expanded there into both
// lanes; sums are FP32 per 256-pixel tile, then FP64.
#include <cmath>
#include <mutex>
#include <type_traits>
#include <vector>

#include <algorithm>

#include "voldor_internal.cuh"

namespace vd {

__device__ __forceinline__ float mufu_rcp(float x)
{
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ float mufu_lg2(float x)
{
    float y;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ float mufu_ex2(float x)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

struct HypF {
    float e0, e1, e2, e3, e4, e5, e6, e7, e8, t0, t1, t2;
};

// log2(1 + r) for r >= 0: below 1/8 r * P(r) with P the degree-3 Chebyshev
// interpolant of log2(1 + r)/r on [0, 1/8] (coefficients highest degree first;
// relative error at most 4.2e-7 in FP32 Horner form, mean 1.9e-7: the nearest
// singularity, r = -1, is seventeen half-widths from the interval, so each
// degree gains a factor ~34); above, lg2(1 + r), an absolute-accuracy
// approximation whose result there is at least log2(9/8) = 0.17. Against the
// earlier degree-4 interpolant on [0, 1/4] this saves one FMA per pair and
// moved the driving window's dense scores by at most 3.1e-8 relative.
constexpr float kL1pC3 = -2.977027297e-01f, kL1pC2 = 4.761879444e-01f, kL1pC1 = -7.212317586e-01f,
                kL1pC0 = 1.442694545e+00f;
constexpr float kL1pMax = 0.125f;

__device__ __forceinline__ float log2_1p_pos(float r)
{
    float s = fmaf(r, kL1pC3, kL1pC2);
    s = fmaf(r, s, kL1pC1);
    s = fmaf(r, s, kL1pC0);
    const float small = r * s;
    const float big = mufu_lg2(1.f + r);
    return r < kL1pMax ? small : big;
}

// Scalar pair term (the allocation-free entry point's form): -ell / ln2 =
// log2(1 + mu/rho) of one (hypothesis, pixel) pair (MIE, Eq. 10), or with kMLE
// log2(r) (MLE, Eq. 9: log rho - log mu = -ln2 * this); behind camera t,
// rho := mu (r = 1). The checked form tests 1 + a_z > 0 and caps the squared
// residual at xs_max.
template <bool kChecked, bool kMLE = false>
__device__ __forceinline__ float pair_term2(const HypF& h, const float4 a, const float4 b, float xs_min, float xs_max)
{
    const float xb = a.x, yb2 = a.y, w = a.z, ut = a.w;
    const float vt = b.x, beta = b.y, beta_k = b.z, Cp = b.w;
    const float ax = fmaf(h.e0, xb, fmaf(h.e1, yb2, fmaf(h.t0, w, h.e2)));
    const float ay = fmaf(h.e3, xb, fmaf(h.e4, yb2, fmaf(h.t1, w, h.e5)));
    const float az = fmaf(h.e6, xb, fmaf(h.e7, yb2, fmaf(h.t2, w, h.e8)));
    const float den = 1.f + az;
    const float rd = mufu_rcp(den);
    const float ru = fmaf(fmaf(-xb, az, ax), rd, -ut);
    const float rv = fmaf(fmaf(-yb2, az, ay), rd, -vt);
    float xs = fmaxf(fmaf(ru, ru, rv * rv), xs_min);
    if (kChecked) xs = fminf(xs, xs_max);
    const float sg = fabsf(fmaf(beta, mufu_lg2(xs), beta_k));
    const float r = Cp * xs * (mufu_ex2(sg) + (2.f + mufu_ex2(-sg)));
    const float v = kMLE ? mufu_lg2(r) : log2_1p_pos(r);
    if (kChecked) return den > 0.f ? v : (kMLE ? 0.f : 1.f);
    return v;
}

// Bulk-copy staging of pixel-record tiles: one thread issues
// cp.async.bulk (global -> shared) completing on an mbarrier per ring slot;
// every thread waits on the slot's phase with a bounded try_wait.
constexpr int kTilePix = 256;                       // records per tile (12 KB)
constexpr int kStages = 2;
constexpr long long kWaitLimit = 1ll << 26;        // bounded spin on an mbarrier phase

__device__ __forceinline__ uint32_t smem_u32(const void* ptr)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(ptr));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(smem_u32(dst)), "l"(src), "r"(bytes), "r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile("{\n .reg .pred P;\n mbarrier.try_wait.parity.shared::cta.b64 P, [%1], %2;\n selp.u32 %0, 1, 0, P;\n}"
                 : "=r"(ok) : "r"(smem_u32(bar)), "r"(parity) : "memory");
    return ok != 0;
}

__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, long long limit = kWaitLimit)
{
    for (long long i = 0; i < limit; ++i)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

// ---------------------------------------------------------------------------
// Packed pair arithmetic (.f32x2) and the packed pair term.
// ---------------------------------------------------------------------------
typedef unsigned long long f2;      // {lo, hi} FP32 lanes

__device__ __forceinline__ f2 f2_pack(float lo, float hi)
{
    f2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}

__device__ __forceinline__ float f2_lo(f2 v)
{
    float lo;
    asm("mov.b64 {%0, _}, %1;" : "=f"(lo) : "l"(v));
    return lo;
}

__device__ __forceinline__ float f2_hi(f2 v)
{
    float hi;
    asm("mov.b64 {_, %0}, %1;" : "=f"(hi) : "l"(v));
    return hi;
}

__device__ __forceinline__ f2 f2_fma(f2 a, f2 b, f2 c)
{
    f2 d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}

__device__ __forceinline__ f2 f2_add(f2 a, f2 b)
{
    f2 d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}

__device__ __forceinline__ f2 f2_sub(f2 a, f2 b)
{
    f2 d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}

__device__ __forceinline__ f2 f2_mul(f2 a, f2 b)
{
    f2 d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}

__device__ __forceinline__ f2 f2_lg2(f2 v) { return f2_pack(mufu_lg2(f2_lo(v)), mufu_lg2(f2_hi(v))); }

// c >= 0 ? a : b, one instruction per lane
__device__ __forceinline__ float slct(float a, float b, float c)
{
    float d;
    asm("slct.f32.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
    return d;
}

// A hypothesis pair in packed form: the rows of a_x and a_y negated, a_z as is.
struct HypX2 {
    f2 x0, x1, x2, xt, y0, y1, y2, yt, z0, z1, z2, zt;
};

// Pixel record expanded in shared memory: each field in both lanes.
struct PixX2 {
    f2 xb, yb2, w, ut, vt, beta, beta_k, Cp, wq, pad;
};
static_assert(sizeof(PixX2) == 80, "PixX2 is five 16-byte words");


// log2(1 + r) (MIE) or log2(r) (MLE), r = mu / rho, of two hypotheses against
// one pixel, with the checks of pair_term2<true>; the residual's sign is
// flipped (it is squared). kGauss: the Gaussian residual model, r = 2^s with
// s = xs fx^2 / alpha - x_mu / alpha (record fields beta, beta_k), and
// log2(1 + 2^s) = max(s, 0) + log2(1 + 2^-|s|).
//
// The term is computed in two halves so that the tile loop can overlap the
// second half of one pixel with the first half of the next: the front
// (projection, reciprocal, squared residual and, under the Fisk model, its
// log2) leaves u = Cp xs, s and -(1 + a_z); the back (the exponentials, the
// log1p and the selects) finishes the term.
struct PairMid {
    f2 u, s, nden;
};

template <bool kGauss>
__device__ __forceinline__ PairMid pair_front(const HypX2& h, const PixX2& q, float xs_min, float xs_max)
{
    const f2 nax = f2_fma(h.x0, q.xb, f2_fma(h.x1, q.yb2, f2_fma(h.xt, q.w, h.x2)));   // -a_x
    const f2 nay = f2_fma(h.y0, q.xb, f2_fma(h.y1, q.yb2, f2_fma(h.yt, q.w, h.y2)));   // -a_y
    const f2 az = f2_fma(h.z0, q.xb, f2_fma(h.z1, q.yb2, f2_fma(h.zt, q.w, h.z2)));
    const f2 mu = f2_fma(q.xb, az, nax);         // xb a_z - a_x
    const f2 mv = f2_fma(q.yb2, az, nay);
    const f2 nden = f2_sub(f2_pack(-1.f, -1.f), az);                     // -(1 + a_z), exactly
    const f2 rd = f2_pack(mufu_rcp(-f2_lo(nden)), mufu_rcp(-f2_hi(nden)));
    const f2 ru = f2_fma(mu, rd, q.ut);          // -(residual u) / fx
    const f2 rv = f2_fma(mv, rd, q.vt);
    f2 xs = f2_fma(ru, ru, f2_mul(rv, rv));
    xs = f2_pack(fminf(fmaxf(f2_lo(xs), xs_min), xs_max), fminf(fmaxf(f2_hi(xs), xs_min), xs_max));
    if (kGauss) return PairMid{xs, f2_fma(q.beta, xs, q.beta_k), nden};       // s = log2(mu / rho)
    return PairMid{f2_mul(q.Cp, xs), f2_fma(q.beta, f2_lg2(xs), q.beta_k), nden};
}

template <bool kMLE, bool kGauss>
__device__ __forceinline__ f2 pair_back(const PairMid& m)
{
    const f2 ONE = f2_pack(1.f, 1.f), TWO = f2_pack(2.f, 2.f);
    const f2 nden = m.nden;
    const float behind = kMLE ? 0.f : 1.f;       // 1 + a_z <= 0: rho := mu
    if (kGauss) {
        const float g0 = f2_lo(m.s), g1 = f2_hi(m.s);
        if (kMLE) return f2_pack(slct(behind, g0, f2_lo(nden)), slct(behind, g1, f2_hi(nden)));
        const f2 e = f2_pack(mufu_ex2(-fabsf(g0)), mufu_ex2(-fabsf(g1)));
        f2 ps = f2_fma(e, f2_pack(kL1pC3, kL1pC3), f2_pack(kL1pC2, kL1pC2));
        ps = f2_fma(e, ps, f2_pack(kL1pC1, kL1pC1));
        ps = f2_fma(e, ps, f2_pack(kL1pC0, kL1pC0));
        const f2 small = f2_mul(e, ps);
        const f2 big = f2_lg2(f2_add(e, ONE));
        const f2 d = f2_add(e, f2_pack(-kL1pMax, -kL1pMax));
        const float v0 = fmaxf(g0, 0.f) + slct(f2_lo(big), f2_lo(small), f2_lo(d));
        const float v1 = fmaxf(g1, 0.f) + slct(f2_hi(big), f2_hi(small), f2_hi(d));
        return f2_pack(slct(behind, v0, f2_lo(nden)), slct(behind, v1, f2_hi(nden)));
    }
    const float s0 = f2_lo(m.s), s1 = f2_hi(m.s);
    const f2 ep = f2_pack(mufu_ex2(s0), mufu_ex2(s1)), en = f2_pack(mufu_ex2(-s0), mufu_ex2(-s1));
    const f2 r = f2_mul(m.u, f2_add(ep, f2_add(en, TWO)));
    if (kMLE) {
        const f2 v = f2_lg2(r);
        return f2_pack(slct(behind, f2_lo(v), f2_lo(nden)), slct(behind, f2_hi(v), f2_hi(nden)));
    }
    f2 ps = f2_fma(r, f2_pack(kL1pC3, kL1pC3), f2_pack(kL1pC2, kL1pC2));
    ps = f2_fma(r, ps, f2_pack(kL1pC1, kL1pC1));
    ps = f2_fma(r, ps, f2_pack(kL1pC0, kL1pC0));
    const f2 small = f2_mul(r, ps);
    const f2 big = f2_lg2(f2_add(r, ONE));
    const f2 d = f2_add(r, f2_pack(-kL1pMax, -kL1pMax));
    const float v0 = slct(f2_lo(big), f2_lo(small), f2_lo(d)), v1 = slct(f2_hi(big), f2_hi(small), f2_hi(d));
    return f2_pack(slct(behind, v0, f2_lo(nden)), slct(behind, v1, f2_hi(nden)));
}

// One shared-memory tile against the first NS hypothesis pairs of the thread,
// software-pipelined over the pixels: the front half of pixel q is issued
// beside the back half of pixel q - 1 (independent chains), and each pixel's
// term is added to the accumulator in pixel order as before.
template <int NS, bool MLE, bool GAUSS>
__device__ __forceinline__ void score_tile(const HypX2* hy, const PixX2* xt, int cnt, float xs_min, float xs_max,
                                           f2* facc)
{
    if (cnt <= 0) return;
    PairMid m[NS];
    f2 wq = xt[0].wq;
#pragma unroll
    for (int k = 0; k < NS; ++k) m[k] = pair_front<GAUSS>(hy[k], xt[0], xs_min, xs_max);
    for (int q = 1; q < cnt; ++q) {
        const PixX2 px = xt[q];
        PairMid n[NS];
#pragma unroll
        for (int k = 0; k < NS; ++k) n[k] = pair_front<GAUSS>(hy[k], px, xs_min, xs_max);
#pragma unroll
        for (int k = 0; k < NS; ++k) {
            facc[k] = f2_fma(wq, pair_back<MLE, GAUSS>(m[k]), facc[k]);
            m[k] = n[k];
        }
        wq = px.wq;
    }
#pragma unroll
    for (int k = 0; k < NS; ++k) facc[k] = f2_fma(wq, pair_back<MLE, GAUSS>(m[k]), facc[k]);
}

// SLOTS hypothesis pairs per thread; MINB resident blocks per SM. A block
// scores a tile of 2 * SLOTS * 256 hypotheses against one chunk of the pixel
// records. The tile is cut into groups of 64 consecutive hypotheses, and warp
// slot k of a warp holds one group, lane l taking hypotheses 2l and 2l + 1 of
// it. A full tile needs every warp slot (16 groups for SLOTS = 2): warp w holds
// groups w * SLOTS .. w * SLOTS + SLOTS - 1 and scores every pixel of the
// chunk. The last, partial tile of a frame needs only u = ceil(m / 64) groups
// for its m hypotheses, i.e. wpg = ceil(u / SLOTS) warps; the block's warps
// then form P = 8 / wpg teams of wpg warps, team j scoring the same groups on
// the j-th of P equal parts of every pixel tile, and the teams' sums are added
// in team order at the end. So a partial tile costs about m / 1024 of a full
// one instead of a whole 512-hypothesis slot per started slot. The autotuner
// picks among the instances.
template <int SLOTS, int MINB, bool MLE, bool GAUSS>
__global__ void __launch_bounds__(kScoreThreads, MINB) k_score(DevParams p, DevState s, int log_idx)
{
    constexpr int HPT = 2 * SLOTS;
    constexpr int kWarps = kScoreThreads / 32;
    const int n_hyp = *s.n_hyp;
    const int n_pix = *s.pix_count;
    if (log_idx >= 0 && blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0) {
        s.score_log[2 * log_idx] = n_hyp;
        s.score_log[2 * log_idx + 1] = n_pix;
    }
    // tile-major block order: the partial last hypothesis tile's (lighter)
    // blocks are scheduled after every full tile's, so they fill the last wave
    const int blk = blockIdx.x + gridDim.x * blockIdx.y;
    const int n_chunks = gridDim.y, chunk = blk % n_chunks;
    const int tile0 = (blk / n_chunks) * (kScoreThreads * HPT);
    if (tile0 >= n_hyp) return;
    const long long lo = (long long)n_pix * chunk / n_chunks;
    const long long hi = (long long)n_pix * (chunk + 1) / n_chunks;
    const int n_tiles = (int)((hi - lo + kTilePix - 1) / kTilePix);

    // work split (block-uniform; warp-uniform per warp)
    const int m = min(n_hyp - tile0, kScoreThreads * HPT);
    const int u = (m + 63) / 64;                       // hypothesis groups of this tile
    const int wpg = (u + SLOTS - 1) / SLOTS;           // warps per team
    const int P = kWarps / wpg;                        // teams
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int team = warp / wpg, wg = warp - team * wpg;
    const int nsw = team < P ? max(0, min(SLOTS, u - wg * SLOTS)) : 0;   // this warp's groups

    __shared__ __align__(128) float4 tile[kStages][kTilePix * 3];
    __shared__ __align__(16) PixX2 xt[kTilePix];
    __shared__ __align__(8) uint64_t full[kStages];
    __shared__ int timed_out;
    const float4* gpix = reinterpret_cast<const float4*>(s.pix);
    auto issue = [&](int it) {
        const long long j0 = lo + (long long)it * kTilePix;
        const int cnt = (int)min((long long)kTilePix, hi - j0);
        const uint32_t bytes = (uint32_t)cnt * (uint32_t)sizeof(PixRec);
        uint64_t* bar = &full[it % kStages];
        mbar_expect_tx(bar, bytes);
        bulk_g2s(&tile[it % kStages][0], gpix + 3 * j0, bytes, bar);
    };
    if (threadIdx.x == 0) {
        for (int i = 0; i < kStages; ++i) mbar_init(&full[i], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        timed_out = 0;
    }
    __syncthreads();
    if (threadIdx.x == 0)
        for (int i = 0; i < kStages && i < n_tiles; ++i) issue(i);

    // hypothesis of slot k, lane half v: tile0 + (wg * SLOTS + k) * 64 + 2 * lane + v
    const int hbase = tile0 + wg * SLOTS * 64 + 2 * lane;
    HypX2 hy[SLOTS];
    {
#pragma unroll
        for (int k = 0; k < SLOTS; ++k) {
            HypF a[2];
#pragma unroll
            for (int v = 0; v < 2; ++v) {
                const int h = hbase + k * 64 + v;
                const float* f = s.hyp_f32 + (size_t)min(h, n_hyp - 1) * 12;
                a[v] = HypF{f[0], f[1], f[2], f[3], f[4], f[5], f[6], f[7], f[8], f[9], f[10], f[11]};
            }
            hy[k] = HypX2{f2_pack(-a[0].e0, -a[1].e0), f2_pack(-a[0].e1, -a[1].e1), f2_pack(-a[0].e2, -a[1].e2),
                          f2_pack(-a[0].t0, -a[1].t0), f2_pack(-a[0].e3, -a[1].e3), f2_pack(-a[0].e4, -a[1].e4),
                          f2_pack(-a[0].e5, -a[1].e5), f2_pack(-a[0].t1, -a[1].t1), f2_pack(a[0].e6, a[1].e6),
                          f2_pack(a[0].e7, a[1].e7), f2_pack(a[0].e8, a[1].e8), f2_pack(a[0].t2, a[1].t2)};
        }
    }
    double acc[HPT];
#pragma unroll
    for (int i = 0; i < HPT; ++i) acc[i] = 0.0;
    const float xs_min = p.xs_min, xs_max = p.xs_max;

    // the tile loop; TEAMS = false is the full-tile case (one team, every
    // pixel), kept as its own copy so that it carries no team state
    int it = 0;
    auto run = [&](auto teams) {
        constexpr bool TEAMS = decltype(teams)::value;
        for (; it < n_tiles; ++it) {
            const int slot = it % kStages;
            if (!mbar_wait_bounded(&full[slot], (uint32_t)((it / kStages) & 1))) atomicExch(&timed_out, 1);
            const int cnt = (int)min((long long)kTilePix, hi - (lo + (long long)it * kTilePix));
            if ((int)threadIdx.x < cnt) {
                // expand record threadIdx.x into both lanes (a timed-out tile's
                // contents are never used)
                const float4* r = &tile[slot][3 * threadIdx.x];
                const float4 a = r[0], b = r[1];
                const float wq = r[2].x;
                float4* x = reinterpret_cast<float4*>(&xt[threadIdx.x]);
                x[0] = make_float4(a.x, a.x, a.y, a.y);
                x[1] = make_float4(a.z, a.z, a.w, a.w);
                x[2] = make_float4(b.x, b.x, b.y, b.y);
                x[3] = make_float4(b.z, b.z, b.w, b.w);
                x[4] = make_float4(wq, wq, 0.f, 0.f);
            }
            __syncthreads();                       // tile expanded; the raw slot is free
            if (timed_out) break;
            if (threadIdx.x == 0 && it + kStages < n_tiles) {
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                issue(it + kStages);
            }
            // this team's part of the tile
            const int q0 = TEAMS ? cnt * team / P : 0, q1 = TEAMS ? cnt * (team + 1) / P : cnt;
            f2 facc[SLOTS];
#pragma unroll
            for (int k = 0; k < SLOTS; ++k) facc[k] = 0ull;
            if (nsw >= SLOTS) score_tile<SLOTS, MLE, GAUSS>(hy, xt + q0, q1 - q0, xs_min, xs_max, facc);
            else if (SLOTS > 3 && nsw == 3) score_tile<(SLOTS > 3 ? 3 : 1), MLE, GAUSS>(hy, xt + q0, q1 - q0, xs_min, xs_max, facc);
            else if (SLOTS > 2 && nsw == 2) score_tile<(SLOTS > 2 ? 2 : 1), MLE, GAUSS>(hy, xt + q0, q1 - q0, xs_min, xs_max, facc);
            else if (nsw == 1) score_tile<1, MLE, GAUSS>(hy, xt + q0, q1 - q0, xs_min, xs_max, facc);
#pragma unroll
            for (int k = 0; k < SLOTS; ++k) {
                acc[2 * k] += (double)f2_lo(facc[k]);
                acc[2 * k + 1] += (double)f2_hi(facc[k]);
            }
            __syncthreads();                       // every thread is done with the expanded tile
        }
    };
    if (P == 1) run(std::false_type{});
    else run(std::true_type{});
    if (timed_out) {
        // drain the copies this block issued (bounded) before leaving
        if (threadIdx.x == 0) {
            for (int j = it; j < n_tiles && j < it + kStages; ++j)
                mbar_wait_bounded(&full[j % kStages], (uint32_t)((j / kStages) & 1));
            atomicOr(s.status + 3, kStatusTimeout);
        }
        return;
    }
    const int S = p.S;
    if (P == 1) {
        if (team == 0) {                               // warps past the one team scored nothing
#pragma unroll
            for (int i = 0; i < HPT; ++i) {
                const int h = hbase + (i >> 1) * 64 + (i & 1);
                if (h < n_hyp) s.partial[(size_t)chunk * S + h] = -acc[i] * 0.69314718055994531;
            }
        }
        return;
    }
    // teams: sums per (team, hypothesis of the tile) in the expanded-tile
    // buffer (free after the loop's last barrier; P * wpg * SLOTS * 64 <=
    // 8 * SLOTS * 64 doubles fit in it), then added in team order
    double* red = reinterpret_cast<double*>(xt);
    const int span = wpg * SLOTS * 64;                 // hypotheses a team covers (>= m)
    static_assert(kWarps * SLOTS * 64 * sizeof(double) <= sizeof(PixX2) * kTilePix, "team sums fit");
    if (team < P) {
#pragma unroll
        for (int i = 0; i < HPT; ++i) red[team * span + (hbase - tile0) + (i >> 1) * 64 + (i & 1)] = acc[i];
    }
    __syncthreads();
    for (int i = threadIdx.x; i < m; i += kScoreThreads) {
        double t = 0.0;
        for (int j = 0; j < P; ++j) t += red[j * span + i];
        s.partial[(size_t)chunk * S + tile0 + i] = -t * 0.69314718055994531;
    }
}

// L_h = sum over the chunks' partials (natural-log units) in a fixed order:
// 32 threads per hypothesis each add a contiguous range of chunks in chunk
// order (loads issued four at a time, so a thread waits on memory about three
// times rather than once per chunk), then their 32 sums are added in range
// order (deterministic). A block covers 32 consecutive hypotheses, so every
// warp's loads are 256 contiguous bytes.
constexpr int kReduceSplit = 32;

__global__ void __launch_bounds__(32 * kReduceSplit) k_score_reduce(DevParams p, DevState s)
{
    __shared__ double part[kReduceSplit][32];
    const int hl = threadIdx.x & 31, q = threadIdx.x >> 5;
    const int h = blockIdx.x * 32 + hl;
    const int n_hyp = *s.n_hyp, nc = s.n_chunks;
    const int c0 = nc * q / kReduceSplit, c1 = nc * (q + 1) / kReduceSplit;
    double v = 0.0;
    if (h < n_hyp) {
        const double* src = s.partial + h;
        const size_t S = (size_t)p.S;
        int c = c0;
        for (; c + 4 <= c1; c += 4) {
            const double a0 = src[(size_t)c * S], a1 = src[(size_t)(c + 1) * S];
            const double a2 = src[(size_t)(c + 2) * S], a3 = src[(size_t)(c + 3) * S];
            v += a0;
            v += a1;
            v += a2;
            v += a3;
        }
        for (; c < c1; ++c) v += src[(size_t)c * S];
    }
    part[q][hl] = v;
    __syncthreads();
    if (q == 0 && h < n_hyp) {
        double t = 0.0;
        for (int r = 0; r < kReduceSplit; ++r) t += part[r][hl];
        s.scores[h] = t;
    }
}

static int g_num_sms = 0;

static int num_sms()
{
    if (g_num_sms == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        if (cudaDeviceGetAttribute(&g_num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || g_num_sms <= 0)
            g_num_sms = 152;
    }
    return g_num_sms;
}

// Pixel chunks so that (hypothesis tiles x chunks) blocks fill `waves` waves
// of the resident blocks of a tile shape.
int score_chunks_for(int S, int N, int hpt, int waves)
{
    const int minb = hpt == 8 ? 1 : (hpt == 4 ? 2 : 3);
    const int tiles = (S + kScoreThreads * hpt - 1) / (kScoreThreads * hpt);
    int chunks = (num_sms() * minb * waves + tiles - 1) / tiles;
    if (chunks > N) chunks = N;
    return chunks < 1 ? 1 : chunks;
}

int score_chunks(int S, int N) { return score_chunks_for(S, N, kScoreDefaultHpt, kScoreDefaultWaves); }

int score_chunks_max(int S, int N)
{
    const int a = score_chunks_for(S, N, 8, kTuneMaxWaves), b = score_chunks_for(S, N, 4, kTuneMaxWaves);
    const int c = score_chunks_for(S, N, 2, kTuneMaxWaves);
    return std::max(a, std::max(b, c));
}

template <int SLOTS, int MINB>
static void launch_score_shape(const DevParams& p, const DevState& s, int li, cudaStream_t st)
{
    dim3 grid((p.S + kScoreThreads * 2 * SLOTS - 1) / (kScoreThreads * 2 * SLOTS), s.n_chunks);
    const bool mle = p.criterion == VOLDOR_CRITERION_MLE, gauss = p.residual == VOLDOR_RESIDUAL_GAUSSIAN;
    if (gauss) {
        if (mle) k_score<SLOTS, MINB, true, true><<<grid, kScoreThreads, 0, st>>>(p, s, li);
        else k_score<SLOTS, MINB, false, true><<<grid, kScoreThreads, 0, st>>>(p, s, li);
    } else {
        if (mle) k_score<SLOTS, MINB, true, false><<<grid, kScoreThreads, 0, st>>>(p, s, li);
        else k_score<SLOTS, MINB, false, false><<<grid, kScoreThreads, 0, st>>>(p, s, li);
    }
}

void launch_score(const DevParams& p, const DevState& s, int log_idx, cudaStream_t st)
{
    const int li = log_idx < kScoreLogMax ? log_idx : -1;
    if (s.score_hpt == 4) launch_score_shape<2, 2>(p, s, li, st);
    else if (s.score_hpt == 2) launch_score_shape<1, 3>(p, s, li, st);
    else launch_score_shape<4, 1>(p, s, li, st);
}

void launch_score_reduce(const DevParams& p, const DevState& s, cudaStream_t st)
{
    k_score_reduce<<<(p.S + 31) / 32, 32 * kReduceSplit, 0, st>>>(p, s);
}


// ---------------------------------------------------------------------------
// Allocation-free dense scoring.
//
// Some callers cannot allocate device memory at the time they want a score:
// code running inside a CUDA stream capture that must not add allocation
// nodes, a host that hands the GPU to this library under a fixed memory
// budget, or a caller whose own allocator owns all device memory. For them,
// voldor_score_records_noalloc scores caller-given pixel records against
// caller-given hypotheses with the same per-pair arithmetic as k_score and
// takes its only scratch (the per-chunk partial sums) from the file-scope
// array below, which every GPU that loads this library holds until the
// process exits.
// ---------------------------------------------------------------------------
constexpr int kStaticMaxHyps = 8192;
constexpr int kStaticChunks = 64;
static __device__ __align__(256) double g_static_partials[kStaticChunks * kStaticMaxHyps];   // 4 MiB

__global__ void __launch_bounds__(kScoreThreads, kScoreBlocksPerSM)
k_score_records(const float4* __restrict__ pix, int n_pix, const float* __restrict__ hyps, int n_hyp, float xs_min,
                float xs_max, double* __restrict__ partial)
{
    const int tile0 = blockIdx.x * kScoreHypsPerBlock;
    if (tile0 >= n_hyp) return;
    const int chunk = blockIdx.y, n_chunks = gridDim.y;
    const long long lo = (long long)n_pix * chunk / n_chunks;
    const long long hi = (long long)n_pix * (chunk + 1) / n_chunks;
    HypF hy[kScoreHypsPerThread];
#pragma unroll
    for (int i = 0; i < kScoreHypsPerThread; ++i) {
        const float* f = hyps + (size_t)min(tile0 + i * kScoreThreads + (int)threadIdx.x, n_hyp - 1) * 12;
        hy[i] = HypF{f[0], f[1], f[2], f[3], f[4], f[5], f[6], f[7], f[8], f[9], f[10], f[11]};
    }
    double acc[kScoreHypsPerThread];
    float facc[kScoreHypsPerThread];
#pragma unroll
    for (int i = 0; i < kScoreHypsPerThread; ++i) { acc[i] = 0.0; facc[i] = 0.f; }
    long long j = lo;
    while (j < hi) {
        const long long jend = min(hi, j + 32);
        for (; j < jend; ++j) {
            const float4 a = __ldg(pix + 3 * j);
            const float4 b = __ldg(pix + 3 * j + 1);
            const float wq = __ldg(reinterpret_cast<const float*>(pix + 3 * j + 2));
#pragma unroll
            for (int i = 0; i < kScoreHypsPerThread; ++i)
                facc[i] = fmaf(wq, pair_term2<true>(hy[i], a, b, xs_min, xs_max), facc[i]);
        }
#pragma unroll
        for (int i = 0; i < kScoreHypsPerThread; ++i) { acc[i] += (double)facc[i]; facc[i] = 0.f; }
    }
#pragma unroll
    for (int i = 0; i < kScoreHypsPerThread; ++i) {
        const int h = tile0 + i * kScoreThreads + threadIdx.x;
        if (h < n_hyp) partial[(size_t)chunk * kStaticMaxHyps + h] = -acc[i] * 0.69314718055994531;
    }
}

__global__ void k_reduce_records(const double* __restrict__ partial, int n_hyp, int n_chunks, double* __restrict__ L)
{
    const int h = blockIdx.x * blockDim.x + threadIdx.x;
    if (h >= n_hyp) return;
    double v = 0.0;
    for (int c = 0; c < n_chunks; ++c) v += partial[(size_t)c * kStaticMaxHyps + h];
    L[h] = v;
}

// Device address of g_static_partials, looked up once per device with that
// device current (a host-side reference to the array is only a stand-in).
constexpr int kStaticMaxDevices = 64;
static double* g_static_ptr[kStaticMaxDevices];
static std::mutex g_static_mutex;

static cudaError_t static_partials(double** out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kStaticMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_static_mutex);
    if (!g_static_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_static_partials);
        if (e != cudaSuccess) return e;
        g_static_ptr[dev] = static_cast<double*>(p);
    }
    *out = g_static_ptr[dev];
    return cudaSuccess;
}

}  // namespace vd

extern "C" voldor_status voldor_score_records_noalloc(const float* records, int n_pix, const float* hyps, int n_hyps,
                                                      double xs_min, double xs_max, double* L, void* cuda_stream)
{
    using namespace vd;
    if (!records || !hyps || !L || n_pix < 0 || n_hyps < 1) return VOLDOR_ERR_INVALID_ARG;
    if (n_hyps > kStaticMaxHyps) return VOLDOR_ERR_INVALID_ARG;
    // the kernel reads records as float4 and writes L as double
    if (((uintptr_t)records & 15u) || ((uintptr_t)hyps & 3u) || ((uintptr_t)L & 7u)) return VOLDOR_ERR_INVALID_ARG;
    if (!(xs_min > 0.0) || !(xs_max > xs_min) || !std::isfinite(xs_max)) return VOLDOR_ERR_INVALID_ARG;
    double* partial = nullptr;
    if (static_partials(&partial) != cudaSuccess) {
        cudaGetLastError();
        return VOLDOR_ERR_CUDA;
    }
    cudaStream_t st = (cudaStream_t)cuda_stream;
    const int tiles = (n_hyps + kScoreHypsPerBlock - 1) / kScoreHypsPerBlock;
    k_score_records<<<dim3(tiles, kStaticChunks), kScoreThreads, 0, st>>>(
        reinterpret_cast<const float4*>(records), n_pix, hyps, n_hyps, (float)xs_min, (float)xs_max, partial);
    k_reduce_records<<<(n_hyps + 255) / 256, 256, 0, st>>>(partial, n_hyps, kStaticChunks, L);
    if (cudaGetLastError() != cudaSuccess) return VOLDOR_ERR_CUDA;
    return VOLDOR_OK;
}

// ---------------------------------------------------------------------------
// Diagnostic: SFU (MUFU) throughput of this GPU in results per SM clock, for
// the roofline of the dense scoring. One wave of blocks (4 per SM, 256
// threads) runs 16 independent chains of one SFU op per thread; the whole
// grid is timed with CUDA events, and the SM clock during the run is measured
// in the kernel (clock64 cycles over globaltimer nanoseconds of each block,
// median over blocks), so results per SM clock = results / (grid time x SM
// clock x SMs) holds at whatever clock the GPU ran.
// ---------------------------------------------------------------------------
namespace vd {
constexpr int kProbeChains = 16;

// One SFU op per chain step, fixed at compile time: with the op chosen at run
// time inside the loop the compiler predicates the branches and issues every
// branch's SFU instruction on each step.
template <int OP>
__device__ __forceinline__ float sfu_step(float v)
{
    float y;
    if constexpr (OP == 0) {          // exp2(-|v|): stays in [0.5, 1)
        asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(-fabsf(v)));
    } else if constexpr (OP == 1) {   // log2(v) + 1.5: converges to ~3.2, stays normal
        asm volatile("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(v));
        y += 1.5f;
    } else {                          // 1 / (-v): alternates between two normal values
        asm volatile("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(-v));
    }
    return y;
}

__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

template <int OP>
__global__ void __launch_bounds__(256) k_sfu_probe(int iters, float seed, float* sink, long long* clk)
{
    float v[kProbeChains];
#pragma unroll
    for (int i = 0; i < kProbeChains; ++i) v[i] = seed + 0.001f * (float)((threadIdx.x + i) & 63);
    __syncthreads();
    const long long c0 = clock64();
    const unsigned long long g0 = global_ns();
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int i = 0; i < kProbeChains; ++i) v[i] = sfu_step<OP>(v[i]);
    }
    __syncthreads();
    const long long c1 = clock64();
    const unsigned long long g1 = global_ns();
    float acc = 0.f;
#pragma unroll
    for (int i = 0; i < kProbeChains; ++i) acc += v[i];
    if (acc == 1234.5f) sink[threadIdx.x] = acc;     // keeps the chains alive
    if (threadIdx.x == 0) {
        clk[2 * blockIdx.x] = c1 - c0;
        clk[2 * blockIdx.x + 1] = (long long)(g1 - g0);
    }
}

void launch_sfu_probe(int op, int blocks, int threads, int iters, float seed, float* sink, long long* clk)
{
    if (op == 0) k_sfu_probe<0><<<blocks, threads>>>(iters, seed, sink, clk);
    else if (op == 1) k_sfu_probe<1><<<blocks, threads>>>(iters, seed, sink, clk);
    else k_sfu_probe<2><<<blocks, threads>>>(iters, seed, sink, clk);
}
}  // namespace vd

extern "C" voldor_status voldor_probe_sfu_rate(int op, double* results_per_sm_clock, double* sm_mhz)
{
    using namespace vd;
    if (!results_per_sm_clock || op < 0 || op > 2) return VOLDOR_ERR_INVALID_ARG;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return VOLDOR_ERR_CUDA;
    const int blocks = sms * 4, threads = 256, iters = 4096;
    float* sink = nullptr;
    long long* clk = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaMalloc(&sink, threads * sizeof(float)) != cudaSuccess) return VOLDOR_ERR_OOM;
    if (cudaMalloc(&clk, 2 * blocks * sizeof(long long)) != cudaSuccess) { cudaFree(sink); return VOLDOR_ERR_OOM; }
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    const float seed = op == 1 ? 1.5f : 0.75f;
    float ms = 0.f;
    std::vector<long long> h(2 * blocks);
    if (e == cudaSuccess) {
        launch_sfu_probe(op, blocks, threads, 256, seed, sink, clk);          // warm-up
        cudaEventRecord(e0);
        launch_sfu_probe(op, blocks, threads, iters, seed, sink, clk);
        cudaEventRecord(e1);
        e = cudaEventSynchronize(e1);
    }
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e == cudaSuccess) e = cudaMemcpy(h.data(), clk, h.size() * sizeof(long long), cudaMemcpyDeviceToHost);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(sink);
    cudaFree(clk);
    if (e != cudaSuccess || !(ms > 0.f)) return VOLDOR_ERR_CUDA;
    std::vector<double> mhz;
    for (int b = 0; b < blocks; ++b)
        if (h[2 * b + 1] > 0) mhz.push_back(1e3 * (double)h[2 * b] / (double)h[2 * b + 1]);
    if (mhz.empty()) return VOLDOR_ERR_INTERNAL;
    std::nth_element(mhz.begin(), mhz.begin() + mhz.size() / 2, mhz.end());
    const double f = mhz[mhz.size() / 2];                      // MHz
    const double results = (double)blocks * threads * (double)kProbeChains * iters;
    *results_per_sm_clock = results / ((double)ms * 1e-3 * f * 1e6 * sms);
    if (sm_mhz) *sm_mhz = f;
    return VOLDOR_OK;
}

// ---------------------------------------------------------------------------
// Diagnostic: the expiry path of the bounded mbarrier waits.
// ---------------------------------------------------------------------------
namespace vd {
// Bounded-wait probe: every thread of one block waits, with the scoring
// kernel's bounded wait, on the first phase of an mbarrier that nothing
// arrives on, for `polls` polls; out[0] = number of threads that gave up,
// out[1] = SM cycles the wait took on thread 0.
__global__ void k_wait_probe(long long polls, long long* out)
{
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    const long long t0 = clock64();
    const bool done = mbar_wait_bounded(&bar, 0, polls);
    const long long t1 = clock64();
    const int gave_up = __syncthreads_count(!done);
    if (threadIdx.x == 0) {
        out[0] = gave_up;
        out[1] = t1 - t0;
    }
}

}  // namespace vd

extern "C" voldor_status voldor_probe_bounded_wait(long long polls, long long* cycles)
{
    using namespace vd;
    if (polls < 0 || polls > kWaitLimit) return VOLDOR_ERR_INVALID_ARG;
    long long* d = nullptr;
    if (cudaMalloc(&d, 2 * sizeof(long long)) != cudaSuccess) return VOLDOR_ERR_OOM;
    k_wait_probe<<<1, 128>>>(polls, d);
    long long h[2] = {0, 0};
    const cudaError_t e = cudaMemcpy(h, d, sizeof(h), cudaMemcpyDeviceToHost);
    cudaFree(d);
    if (e != cudaSuccess || cudaGetLastError() != cudaSuccess) return VOLDOR_ERR_CUDA;
    if (cycles) *cycles = h[1];
    return h[0] == 128 ? VOLDOR_ERR_TIMEOUT : (h[0] == 0 ? VOLDOR_OK : VOLDOR_ERR_INTERNAL);
}

