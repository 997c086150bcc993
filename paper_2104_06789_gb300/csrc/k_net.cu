// Learned depth / rigidness proposal: a 6-layer 3x3 convolutional network
// (2T -> 32 -> 32 -> 32 -> 32 -> 32 -> 2, ReLU between layers) that reads the
// flow stack of a window and predicts, per pixel of I_0, a log-depth and a
// rigidness logit used in place of the triangulation bootstrap. BF16
// activations and weights, FP32 accumulation, tensor cores (mma.sync
// m16n8k16 with ldmatrix operand loads) for the forward pass, the input
// gradient and the weight gradient; FP32 Adam on master weights.
//
// Input: the flows of each frame divided by that frame's mean flow magnitude
// (the network sees the shape of the flow field, not its overall size).
// Output scale: a network reading 3x3 neighbourhoods of flows cannot know the
// translation's magnitude, so it is trained on log-depth relative to the
// window's median; the learned bootstrap restores the metric scale fixed by
// the given T_1 by shifting the prediction to the median log-ratio against the
// triangulated depth (a two-level histogram median on the device).
//
// Layouts: activations NHWC bf16 with a channel stride of 16 (input) or 32;
// weights per layer [Cout_pad][9][Cin_pad] bf16 (tap = 3 ky + kx), and for the
// input gradient the flipped transpose [Cin_pad][9][Cout_pad]; master
// parameters FP32 [Cout][9][Cin] then bias[Cout] per layer.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include <cuda_bf16.h>

#include "voldor_internal.cuh"

namespace vd {

typedef __nv_bfloat16 bf16;

constexpr int kNetLayers = 6;
constexpr int kNetWidth = 32;
constexpr int kTileW = 32, kTileH = 4;          // block tile: 4 rows of 32 pixels, one row per warp
constexpr int kHaloW = kTileW + 2, kHaloH = kTileH + 2;
constexpr int kAlignBins = 2048;                // histogram bins per level of the median search
constexpr float kAlignRange = 16.f;             // first level covers log-ratios in [-16, 16)

__device__ __forceinline__ uint32_t smem_addr(const void* p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void ldsm_x4(uint32_t addr, uint32_t& r0, uint32_t& r1, uint32_t& r2, uint32_t& r3)
{
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3) : "r"(addr));
}

__device__ __forceinline__ void ldsm_x4_t(uint32_t addr, uint32_t& r0, uint32_t& r1, uint32_t& r2, uint32_t& r3)
{
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3) : "r"(addr));
}

__device__ __forceinline__ void ldsm_x2(uint32_t addr, uint32_t& r0, uint32_t& r1)
{
    asm volatile("ldmatrix.sync.aligned.m8n8.x2.shared.b16 {%0,%1}, [%2];" : "=r"(r0), "=r"(r1) : "r"(addr));
}

__device__ __forceinline__ void ldsm_x2_t(uint32_t addr, uint32_t& r0, uint32_t& r1)
{
    asm volatile("ldmatrix.sync.aligned.m8n8.x2.trans.shared.b16 {%0,%1}, [%2];" : "=r"(r0), "=r"(r1) : "r"(addr));
}

__device__ __forceinline__ void mma_bf16(float* c, uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3, uint32_t b0,
                                         uint32_t b1)
{
    asm volatile("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
                 "{%0,%1,%2,%3};"
                 : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
                 : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// Loads the (kTileH + 2) x (kTileW + 2) input halo of a tile, CIN channels per
// pixel (global channel stride cin_g), zero outside the image.
template <int CIN, int CS>
__device__ __forceinline__ void load_halo(bf16* s, const bf16* in, int cin_g, int H, int W, int b, int x0, int y0)
{
    constexpr int VEC = CIN / 8;   // 16-byte vectors per pixel
    for (int i = threadIdx.x; i < kHaloH * kHaloW * VEC; i += blockDim.x) {
        const int q = i / VEC, v = i % VEC;
        const int gy = y0 + q / kHaloW - 1, gx = x0 + q % kHaloW - 1;
        uint4 val = make_uint4(0, 0, 0, 0);
        if (gy >= 0 && gy < H && gx >= 0 && gx < W)
            val = *reinterpret_cast<const uint4*>(in + (((size_t)b * H + gy) * W + gx) * cin_g + v * 8);
        *reinterpret_cast<uint4*>(s + q * CS + v * 8) = val;
    }
}

// ---------------------------------------------------------------------------
// 3x3 convolution (implicit GEMM): out[p][n] = sum_{tap, c} in[p + off(tap)][c]
// w[n][tap][c] (+ bias[n]), for NT*8 output channels. Each warp computes one
// tile row of 32 pixels as two m16 tiles; K runs over 9 taps x CIN channels in
// k16 steps. Epilogue: optional bias, ReLU, and the ReLU mask of a previous
// activation (for the input gradient); bf16 or fp32 output.
// ---------------------------------------------------------------------------
struct ConvArgs {
    const bf16* in;
    int cin_g;
    const bf16* w;          // [NT*8][9][CIN] bf16
    const float* bias;      // NT*8 or null
    bf16* out;              // bf16 output (channel stride cout_g) or null
    float* out_f;           // fp32 output (channel stride cout_g) or null
    int cout_g;
    int n_out;              // real output channels written
    const bf16* mask;       // zero the output where mask <= 0 (channel stride cout_g), or null
    int relu;
    int H, W;
};

template <int CIN, int NT>
__global__ void __launch_bounds__(128) k_conv3x3(ConvArgs a)
{
    constexpr int CS = CIN + 8;                 // padded pixel stride (bank-conflict free)
    constexpr int WS = 9 * CIN + 8;             // padded weight row stride
    __shared__ __align__(16) bf16 in_s[kHaloH * kHaloW * CS];
    __shared__ __align__(16) bf16 w_s[NT * 8 * WS];
    const int x0 = blockIdx.x * kTileW, y0 = blockIdx.y * kTileH, b = blockIdx.z;
    for (int i = threadIdx.x; i < NT * 8 * (9 * CIN / 8); i += blockDim.x) {
        const int n = i / (9 * CIN / 8), v = i % (9 * CIN / 8);
        *reinterpret_cast<uint4*>(w_s + n * WS + v * 8) = *reinterpret_cast<const uint4*>(a.w + (size_t)n * 9 * CIN + v * 8);
    }
    load_halo<CIN, CS>(in_s, a.in, a.cin_g, a.H, a.W, b, x0, y0);
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int gid = lane >> 2, tig = lane & 3;
    for (int mt = 0; mt < 2; ++mt) {
        float acc[NT][4];
#pragma unroll
        for (int n = 0; n < NT; ++n) acc[n][0] = acc[n][1] = acc[n][2] = acc[n][3] = 0.f;
#pragma unroll
        for (int tap = 0; tap < 9; ++tap) {
            const int ky = tap / 3, kx = tap % 3;
#pragma unroll
            for (int kc = 0; kc < CIN / 16; ++kc) {
                uint32_t a0, a1, a2, a3;
                const int px = mt * 16 + (lane & 15) + kx;
                ldsm_x4(smem_addr(in_s + ((warp + ky) * kHaloW + px) * CS + kc * 16 + (lane >> 4) * 8), a0, a1, a2, a3);
#pragma unroll
                for (int n = 0; n < NT; ++n) {
                    uint32_t b0, b1;
                    ldsm_x2(smem_addr(w_s + (n * 8 + (lane & 7)) * WS + tap * CIN + kc * 16 + ((lane >> 3) & 1) * 8), b0, b1);
                    mma_bf16(acc[n], a0, a1, a2, a3, b0, b1);
                }
            }
        }
        const int py = y0 + warp;
#pragma unroll
        for (int n = 0; n < NT; ++n) {
#pragma unroll
            for (int half = 0; half < 2; ++half) {
                const int px = x0 + mt * 16 + gid + 8 * half;
                if (py >= a.H || px >= a.W) continue;
                const int co = n * 8 + 2 * tig;
                const size_t o = (((size_t)b * a.H + py) * a.W + px) * a.cout_g + co;
                float v0 = acc[n][2 * half], v1 = acc[n][2 * half + 1];
                if (a.bias) { v0 += a.bias[co]; v1 += a.bias[co + 1]; }
                if (a.relu) { v0 = fmaxf(v0, 0.f); v1 = fmaxf(v1, 0.f); }
                if (a.mask) {
                    if (!(__bfloat162float(a.mask[o]) > 0.f)) v0 = 0.f;
                    if (!(__bfloat162float(a.mask[o + 1]) > 0.f)) v1 = 0.f;
                }
                if (a.out) {
                    if (co < a.n_out) a.out[o] = __float2bfloat16_rn(v0);
                    if (co + 1 < a.n_out) a.out[o + 1] = __float2bfloat16_rn(v1);
                }
                if (a.out_f) {
                    if (co < a.n_out) a.out_f[o] = v0;
                    if (co + 1 < a.n_out) a.out_f[o + 1] = v1;
                }
            }
        }
    }
}

// ---------------------------------------------------------------------------
// Weight gradient: dw[co][tap][ci] += sum_p dout[p][co] in[p + off(tap)][ci],
// db[co] += sum_p dout[p][co]. GEMM with M = output channels (MT m16 tiles),
// N = CIN, K = pixels of `tiles` consecutive spatial tiles per block; warp w
// owns taps w, w+4, w+8. Operands come from shared memory with transposing
// ldmatrix (both are stored pixel-major). FP32 atomics into dw at the end.
// ---------------------------------------------------------------------------
struct WgradArgs {
    const bf16* in;
    int cin_g;
    const bf16* dout;       // channel stride cout_g
    int cout_g;
    float* dw;              // [n_out][9][cin_real]
    float* db;              // [n_out]
    int n_out, cin_real;
    int H, W, B;
    int tiles_x, tiles_y;
    int tiles_per_block;
};

template <int CIN, int MT>
__global__ void __launch_bounds__(128) k_conv_wgrad(WgradArgs a)
{
    constexpr int CS = CIN + 8;
    constexpr int OS = MT * 16 + 8;             // dout pixel stride in shared memory
    constexpr int NT = CIN / 8;
    __shared__ __align__(16) bf16 in_s[kHaloH * kHaloW * CS];
    __shared__ __align__(16) bf16 do_s[kTileH * kTileW * OS];
    __shared__ float db_s[MT * 16];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int gid = lane >> 2, tig = lane & 3;
    float acc[3][MT][NT][4];
#pragma unroll
    for (int ti = 0; ti < 3; ++ti)
#pragma unroll
        for (int m = 0; m < MT; ++m)
#pragma unroll
            for (int n = 0; n < NT; ++n) acc[ti][m][n][0] = acc[ti][m][n][1] = acc[ti][m][n][2] = acc[ti][m][n][3] = 0.f;
    if (threadIdx.x < MT * 16) db_s[threadIdx.x] = 0.f;
    const int total_tiles = a.tiles_x * a.tiles_y * a.B;
    for (int tt = 0; tt < a.tiles_per_block; ++tt) {
        const int tile = blockIdx.x * a.tiles_per_block + tt;
        if (tile >= total_tiles) break;
        const int b = tile / (a.tiles_x * a.tiles_y);
        const int rem = tile % (a.tiles_x * a.tiles_y);
        const int x0 = (rem % a.tiles_x) * kTileW, y0 = (rem / a.tiles_x) * kTileH;
        __syncthreads();
        load_halo<CIN, CS>(in_s, a.in, a.cin_g, a.H, a.W, b, x0, y0);
        for (int i = threadIdx.x; i < kTileH * kTileW * (MT * 2); i += blockDim.x) {
            const int q = i / (MT * 2), v = i % (MT * 2);
            const int gy = y0 + q / kTileW, gx = x0 + q % kTileW;
            uint4 val = make_uint4(0, 0, 0, 0);
            if (gy < a.H && gx < a.W)
                val = *reinterpret_cast<const uint4*>(a.dout + (((size_t)b * a.H + gy) * a.W + gx) * a.cout_g + v * 8);
            *reinterpret_cast<uint4*>(do_s + q * OS + v * 8) = val;
        }
        __syncthreads();
        if (threadIdx.x < a.n_out) {
            float sdb = 0.f;
            for (int q = 0; q < kTileH * kTileW; ++q) sdb += __bfloat162float(do_s[q * OS + threadIdx.x]);
            db_s[threadIdx.x] += sdb;
        }
        // K steps: 16 consecutive pixels of one tile row
        for (int ks = 0; ks < kTileH * kTileW / 16; ++ks) {
            const int r = ks >> 1, h = ks & 1;
            uint32_t af[MT][4];
#pragma unroll
            for (int m = 0; m < MT; ++m) {
                const int k = (lane & 7) + ((lane >> 4) << 3);
                const int moff = ((lane >> 3) & 1) << 3;
                ldsm_x4_t(smem_addr(do_s + (r * kTileW + h * 16 + k) * OS + m * 16 + moff), af[m][0], af[m][1], af[m][2],
                          af[m][3]);
            }
#pragma unroll
            for (int ti = 0; ti < 3; ++ti) {
                const int tap = warp + 4 * ti;
                if (tap >= 9) break;
                const int ky = tap / 3, kx = tap % 3;
#pragma unroll
                for (int n = 0; n < NT; ++n) {
                    uint32_t b0, b1;
                    const int k = lane & 15;
                    ldsm_x2_t(smem_addr(in_s + ((r + ky) * kHaloW + h * 16 + k + kx) * CS + n * 8), b0, b1);
#pragma unroll
                    for (int m = 0; m < MT; ++m) mma_bf16(acc[ti][m][n], af[m][0], af[m][1], af[m][2], af[m][3], b0, b1);
                }
            }
        }
    }
#pragma unroll
    for (int ti = 0; ti < 3; ++ti) {
        const int tap = warp + 4 * ti;
        if (tap >= 9) break;
#pragma unroll
        for (int m = 0; m < MT; ++m)
#pragma unroll
            for (int n = 0; n < NT; ++n)
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const int co = m * 16 + gid + ((e >> 1) << 3);
                    const int ci = n * 8 + 2 * tig + (e & 1);
                    if (co < a.n_out && ci < a.cin_real) atomicAdd(a.dw + ((size_t)co * 9 + tap) * a.cin_real + ci, acc[ti][m][n][e]);
                }
    }
    __syncthreads();
    if (threadIdx.x < a.n_out) atomicAdd(a.db + threadIdx.x, db_s[threadIdx.x]);
}

// ---------------------------------------------------------------------------
// Input packing, loss, parameter packing, Adam, proposal output.
// ---------------------------------------------------------------------------
// Sum of |flow| per (image, frame): grid (blocks, B*T), one atomic per block.
__global__ void k_flow_norm_sum(const void* flows, int f16, size_t N, float* sums)
{
    const int bt = blockIdx.y;
    float s = 0.f;
    for (size_t p = (size_t)blockIdx.x * blockDim.x + threadIdx.x; p < N; p += (size_t)gridDim.x * blockDim.x) {
        const float2 f = load_flow(flows, f16, (size_t)bt * N + p);
        const float m = sqrtf(f.x * f.x + f.y * f.y);
        s += isfinite(m) ? m : 0.f;
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    __shared__ float ws[32];
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        float t = 0.f;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += ws[w];
        atomicAdd(sums + bt, t);
    }
}

__global__ void k_pack_input(const void* flows, int f16, int T, int H, int W, int B, const float* sums, bf16* in0)
{
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const size_t N = (size_t)H * W;
    if (i >= N * B) return;
    const size_t b = i / N, p = i % N;
    __align__(16) bf16 v[16];
    for (int c = 0; c < 16; ++c) v[c] = __float2bfloat16_rn(0.f);
    for (int t = 0; t < T && t < 8; ++t) {
        const size_t idx = (b * T + t) * N + p;
        const float2 f = load_flow(flows, f16, idx);
        const float s = sums[b * T + t];
        const float inv = s > 0.f ? (float)N / s : 0.f;       // 1 / mean |flow| of the frame
        v[2 * t] = __float2bfloat16_rn(f.x * inv);
        v[2 * t + 1] = __float2bfloat16_rn(f.y * inv);
    }
    uint4* o = reinterpret_cast<uint4*>(in0 + i * 16);
    o[0] = *reinterpret_cast<uint4*>(v);
    o[1] = *reinterpret_cast<uint4*>(v + 8);
}

// Per pixel: Huber loss (delta 0.1) on log-depth, binary cross-entropy on the
// rigidness logit (weight lam_r); gradients into channels 0, 1 of a 16-channel
// bf16 buffer, scaled by 1 / n_pix. Targets with a non-finite log-depth are
// skipped.
__global__ void k_net_loss(const float* pred, int pred_cs, const float* tgt, size_t n_pix, float lam_r, bf16* dout,
                           float* loss)
{
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    float l = 0.f;
    if (i < n_pix) {
        const float z0 = pred[i * pred_cs], z1 = pred[i * pred_cs + 1];
        const float t0 = tgt[2 * i], t1 = tgt[2 * i + 1];
        float g0 = 0.f, g1 = 0.f;
        if (isfinite(t0) && isfinite(z0) && isfinite(z1)) {
            const float d = z0 - t0, ad = fabsf(d), delta = 0.1f;
            l = ad < delta ? 0.5f * d * d / delta : ad - 0.5f * delta;
            g0 = ad < delta ? d / delta : copysignf(1.f, d);
            const float sp = z1 > 0.f ? z1 + log1pf(expf(-z1)) : log1pf(expf(z1));
            l += lam_r * (sp - t1 * z1);
            g1 = lam_r * (1.f / (1.f + expf(-z1)) - t1);
        }
        const float inv = 1.f / (float)n_pix;
        __align__(16) bf16 v[16];
        for (int c = 0; c < 16; ++c) v[c] = __float2bfloat16_rn(0.f);
        v[0] = __float2bfloat16_rn(g0 * inv);
        v[1] = __float2bfloat16_rn(g1 * inv);
        uint4* o = reinterpret_cast<uint4*>(dout + i * 16);
        o[0] = *reinterpret_cast<uint4*>(v);
        o[1] = *reinterpret_cast<uint4*>(v + 8);
    }
    for (int o = 16; o > 0; o >>= 1) l += __shfl_xor_sync(0xffffffffu, l, o);
    if ((threadIdx.x & 31) == 0 && l != 0.f) atomicAdd(loss, l / (float)n_pix);
}

struct NetLayout {
    int cin[kNetLayers], cout[kNetLayers], cin_pad[kNetLayers], cout_pad[kNetLayers];
    size_t w_off[kNetLayers], b_off[kNetLayers];   // into the FP32 master vector
    size_t fw_off[kNetLayers], bw_off[kNetLayers];  // into the bf16 forward / backward weight buffers
    size_t n_params, n_fw, n_bw;
};

static NetLayout net_layout(int T)
{
    NetLayout L;
    size_t p = 0, f = 0, g = 0;
    for (int l = 0; l < kNetLayers; ++l) {
        L.cin[l] = l == 0 ? 2 * T : kNetWidth;
        L.cout[l] = l == kNetLayers - 1 ? 2 : kNetWidth;
        L.cin_pad[l] = l == 0 ? 16 : kNetWidth;
        L.cout_pad[l] = l == kNetLayers - 1 ? 8 : kNetWidth;
        L.w_off[l] = p;
        p += (size_t)L.cout[l] * 9 * L.cin[l];
        L.b_off[l] = p;
        p += L.cout[l];
        L.fw_off[l] = f;
        f += (size_t)L.cout_pad[l] * 9 * L.cin_pad[l];
        // backward weights: [cin_pad][9][cout_bw] with the output side padded to 16
        L.bw_off[l] = g;
        g += (size_t)L.cin_pad[l] * 9 * (L.cout_pad[l] < 16 ? 16 : L.cout_pad[l]);
    }
    L.n_params = p;
    L.n_fw = f;
    L.n_bw = g;
    return L;
}

// FP32 master -> bf16 forward weights [cout_pad][9][cin_pad] and backward
// weights [cin_pad][9][cout_bw] with taps flipped (tap 8 - t), zero padded.
__global__ void k_pack_weights(NetLayout L, const float* master, bf16* fw, bf16* bw, float* fbias)
{
    const int l = blockIdx.y;
    const int cin = L.cin[l], cout = L.cout[l], cinp = L.cin_pad[l], coutp = L.cout_pad[l];
    const int coutb = coutp < 16 ? 16 : coutp;
    const float* Wm = master + L.w_off[l];
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < coutp * 9 * cinp; i += gridDim.x * blockDim.x) {
        const int co = i / (9 * cinp), tap = (i / cinp) % 9, ci = i % cinp;
        const float v = (co < cout && ci < cin) ? Wm[((size_t)co * 9 + tap) * cin + ci] : 0.f;
        fw[L.fw_off[l] + i] = __float2bfloat16_rn(v);
    }
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < cinp * 9 * coutb; i += gridDim.x * blockDim.x) {
        const int ci = i / (9 * coutb), tap = (i / coutb) % 9, co = i % coutb;
        const float v = (co < cout && ci < cin) ? Wm[((size_t)co * 9 + (8 - tap)) * cin + ci] : 0.f;
        bw[L.bw_off[l] + i] = __float2bfloat16_rn(v);
    }
    if (blockIdx.x == 0)
        for (int i = threadIdx.x; i < coutp; i += blockDim.x) fbias[l * kNetWidth + i] = i < cout ? master[L.b_off[l] + i] : 0.f;
}

__global__ void k_adam(float* w, float* m, float* v, const float* g, size_t n, float lr, float b1, float b2, float eps,
                       float c1, float c2)
{
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    w[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

// Scale alignment: median over pixels of log(theta_tri) - z0, where the
// triangulated depth is strictly inside the depth range and z0 is finite.
// Level 0 bins [-16, 16) (values outside go to the end bins); level 1 bins
// the median bin of level 0. align = {lo, hi, rank, shift, count}.
__global__ void k_align_hist(const float* pred, int pred_cs, const float* theta, int N, float d_min, float d_max,
                             const float* align, int level, unsigned* hist)
{
    __shared__ unsigned h[kAlignBins];
    for (int i = threadIdx.x; i < kAlignBins; i += blockDim.x) h[i] = 0;
    __syncthreads();
    const float lo = level == 0 ? -kAlignRange : align[0];
    const float hi = level == 0 ? kAlignRange : align[1];
    const float scale = kAlignBins / (hi - lo);
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < N; j += gridDim.x * blockDim.x) {
        const float th = theta[j], z0 = pred[(size_t)j * pred_cs];
        if (!(th > d_min * 1.0001f && th < d_max * 0.9999f) || !isfinite(z0)) continue;
        const float v = logf(th) - z0;
        if (!isfinite(v)) continue;
        if (level == 1 && !(v >= lo && v < hi)) continue;
        int bin = (int)floorf((v - lo) * scale);
        bin = bin < 0 ? 0 : (bin >= kAlignBins ? kAlignBins - 1 : bin);
        atomicAdd(&h[bin], 1u);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < kAlignBins; i += blockDim.x)
        if (h[i]) atomicAdd(hist + (size_t)level * kAlignBins + i, h[i]);
}

// One thread: picks the bin holding the median (level 0: rank (count-1)/2 of
// all valid values; level 1: the remaining rank inside the chosen bin).
__global__ void k_align_select(const unsigned* hist, int level, float* align)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const unsigned* h = hist + (size_t)level * kAlignBins;
    const float lo = level == 0 ? -kAlignRange : align[0];
    const float hi = level == 0 ? kAlignRange : align[1];
    unsigned long long total = 0;
    for (int i = 0; i < kAlignBins; ++i) total += h[i];
    if (level == 0) {
        align[4] = (float)total;
        if (total == 0) { align[3] = 0.f; align[0] = 0.f; align[1] = 0.f; align[2] = -1.f; return; }
        const unsigned long long rank = (total - 1) / 2;
        unsigned long long cum = 0;
        int bin = 0;
        for (; bin < kAlignBins - 1 && cum + h[bin] <= rank; ++bin) cum += h[bin];
        const float w = (hi - lo) / kAlignBins;
        align[0] = lo + w * bin;
        align[1] = lo + w * (bin + 1);
        // the end bins also hold the clamped out-of-range values: no refinement there
        align[2] = (bin == 0 || bin == kAlignBins - 1) ? -1.f : (float)(rank - cum);
        align[3] = lo + w * (bin + 0.5f);
        return;
    }
    if (align[2] < 0.f || total == 0) return;       // nothing valid, or the median sits in an end bin
    const unsigned long long rank = (unsigned long long)align[2];
    unsigned long long cum = 0;
    int bin = 0;
    for (; bin < kAlignBins - 1 && cum + h[bin] <= rank; ++bin) cum += h[bin];
    const float w = (hi - lo) / kAlignBins;
    align[3] = lo + w * (bin + 0.5f);
}

// Proposal into a window state (either pointer may be null): theta =
// exp(log-depth + shift) clamped to the depth range, W_t = sigmoid(logit).
__global__ void k_net_to_state(const float* pred, int pred_cs, int N, int T, float d_min, float d_max,
                               const float* align, float* theta, float* wmap)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= N) return;
    if (theta) {
        const float z0 = pred[(size_t)j * pred_cs] + align[3];
        float d = expf(fminf(fmaxf(z0, -30.f), 30.f));
        d = fminf(fmaxf(d, d_min), d_max);
        theta[j] = isfinite(d) ? d : d_max;
    }
    if (wmap) {
        const float w = 1.f / (1.f + expf(-pred[(size_t)j * pred_cs + 1]));
        for (int t = 0; t < T; ++t) wmap[(size_t)t * N + j] = isfinite(w) ? w : 1.f;
    }
}

}  // namespace vd

// ---------------------------------------------------------------------------
// Host side: the network object.
// ---------------------------------------------------------------------------
using namespace vd;

struct voldor_net {
    int T = 0;
    NetLayout L{};
    float *master = nullptr, *m = nullptr, *v = nullptr, *grad = nullptr;
    bf16 *fw = nullptr, *bw = nullptr;
    float* fbias = nullptr;
    float* loss = nullptr;
    float* align = nullptr;          // [8] scale alignment state
    unsigned* hist = nullptr;        // [2][kAlignBins]
    float* fsum = nullptr;           // [cap_bt] sum of |flow| per (image, frame)
    size_t cap_bt = 0;
    int step = 0;
    size_t cap_pix = 0;
    bf16* in0 = nullptr;            // [pix][16]
    bf16* act[kNetLayers - 1] = {}; // [pix][32]
    float* pred = nullptr;          // [pix][8]
    bf16* g16 = nullptr;            // [pix][16] gradient at the output
    bf16 *ga = nullptr, *gb = nullptr;   // [pix][32] gradient ping-pong
};

namespace {

bool net_ok(cudaError_t e) { return e == cudaSuccess; }

void net_free_acts(voldor_net* n)
{
    cudaFree(n->in0);
    for (auto& a : n->act) { cudaFree(a); a = nullptr; }
    cudaFree(n->pred);
    cudaFree(n->g16);
    cudaFree(n->ga);
    cudaFree(n->gb);
    n->in0 = nullptr; n->pred = nullptr; n->g16 = nullptr; n->ga = nullptr; n->gb = nullptr;
    n->cap_pix = 0;
}

voldor_status net_reserve(voldor_net* n, size_t pix, size_t bt)
{
    if (bt > n->cap_bt) {
        cudaFree(n->fsum);
        n->fsum = nullptr;
        n->cap_bt = 0;
        if (!net_ok(cudaMalloc(&n->fsum, bt * sizeof(float)))) {
            cudaGetLastError();
            return VOLDOR_ERR_OOM;
        }
        n->cap_bt = bt;
    }
    if (pix <= n->cap_pix) return VOLDOR_OK;
    net_free_acts(n);
    bool ok = net_ok(cudaMalloc(&n->in0, pix * 16 * sizeof(bf16))) && net_ok(cudaMalloc(&n->pred, pix * 8 * sizeof(float))) &&
              net_ok(cudaMalloc(&n->g16, pix * 16 * sizeof(bf16))) && net_ok(cudaMalloc(&n->ga, pix * 32 * sizeof(bf16))) &&
              net_ok(cudaMalloc(&n->gb, pix * 32 * sizeof(bf16)));
    for (auto& a : n->act) ok = ok && net_ok(cudaMalloc(&a, pix * 32 * sizeof(bf16)));
    if (!ok) {
        cudaGetLastError();
        net_free_acts(n);
        return VOLDOR_ERR_OOM;
    }
    n->cap_pix = pix;
    return VOLDOR_OK;
}

void pack(voldor_net* n, cudaStream_t st)
{
    k_pack_weights<<<dim3(32, kNetLayers), 256, 0, st>>>(n->L, n->master, n->fw, n->bw, n->fbias);
}

void conv(int cin_pad, int ntiles, const ConvArgs& a, int B, cudaStream_t st)
{
    dim3 grid((a.W + kTileW - 1) / kTileW, (a.H + kTileH - 1) / kTileH, B);
    if (cin_pad == 16 && ntiles == 4) k_conv3x3<16, 4><<<grid, 128, 0, st>>>(a);
    else if (cin_pad == 32 && ntiles == 4) k_conv3x3<32, 4><<<grid, 128, 0, st>>>(a);
    else if (cin_pad == 32 && ntiles == 1) k_conv3x3<32, 1><<<grid, 128, 0, st>>>(a);
}

// Forward pass of B images of H x W; predictions in n->pred (8 floats per pixel).
void forward(voldor_net* n, const void* flows, int f16, int B, int H, int W, cudaStream_t st)
{
    const size_t pix = (size_t)B * H * W;
    const size_t N = (size_t)H * W;
    cudaMemsetAsync(n->fsum, 0, (size_t)B * n->T * sizeof(float), st);
    const unsigned nb = (unsigned)std::min<size_t>((N + 255) / 256, 64);
    k_flow_norm_sum<<<dim3(nb, B * n->T), 256, 0, st>>>(flows, f16, N, n->fsum);
    k_pack_input<<<(unsigned)((pix + 255) / 256), 256, 0, st>>>(flows, f16, n->T, H, W, B, n->fsum, n->in0);
    const bf16* in = n->in0;
    int cin_g = 16;
    for (int l = 0; l < kNetLayers; ++l) {
        const bool last = l == kNetLayers - 1;
        ConvArgs a{};
        a.in = in; a.cin_g = cin_g; a.w = n->fw + n->L.fw_off[l]; a.bias = n->fbias + l * kNetWidth;
        a.out = last ? nullptr : n->act[l]; a.out_f = last ? n->pred : nullptr;
        a.cout_g = last ? 8 : 32; a.n_out = last ? 8 : 32; a.mask = nullptr; a.relu = last ? 0 : 1; a.H = H; a.W = W;
        conv(n->L.cin_pad[l], n->L.cout_pad[l] / 8, a, B, st);
        if (last) break;
        in = n->act[l];
        cin_g = 32;
    }
}

void wgrad(voldor_net* n, int l, const bf16* in, int cin_g, const bf16* dout, int cout_g, int B, int H, int W, cudaStream_t st)
{
    WgradArgs a{};
    a.in = in; a.cin_g = cin_g; a.dout = dout; a.cout_g = cout_g;
    a.dw = n->grad + n->L.w_off[l]; a.db = n->grad + n->L.b_off[l];
    a.n_out = n->L.cout[l]; a.cin_real = n->L.cin[l];
    a.H = H; a.W = W; a.B = B;
    a.tiles_x = (W + kTileW - 1) / kTileW; a.tiles_y = (H + kTileH - 1) / kTileH;
    const int total = a.tiles_x * a.tiles_y * B;
    a.tiles_per_block = total > 1216 ? (total + 1215) / 1216 : 1;
    const int blocks = (total + a.tiles_per_block - 1) / a.tiles_per_block;
    const int cinp = n->L.cin_pad[l];
    const int mt = n->L.cout[l] > 16 ? 2 : 1;
    if (cinp == 16 && mt == 2) k_conv_wgrad<16, 2><<<blocks, 128, 0, st>>>(a);
    else if (cinp == 32 && mt == 2) k_conv_wgrad<32, 2><<<blocks, 128, 0, st>>>(a);
    else if (cinp == 32 && mt == 1) k_conv_wgrad<32, 1><<<blocks, 128, 0, st>>>(a);
}

// Backward pass after forward(); target [pix][2] (log-depth, rigidness).
void backward(voldor_net* n, const float* tgt, int B, int H, int W, float lam_r, cudaStream_t st)
{
    const size_t pix = (size_t)B * H * W;
    cudaMemsetAsync(n->grad, 0, n->L.n_params * sizeof(float), st);
    cudaMemsetAsync(n->loss, 0, sizeof(float), st);
    k_net_loss<<<(unsigned)((pix + 255) / 256), 256, 0, st>>>(n->pred, 8, tgt, pix, lam_r, n->g16, n->loss);
    const bf16* dout = n->g16;
    int dout_g = 16;
    bf16* bufs[2] = {n->ga, n->gb};
    for (int l = kNetLayers - 1; l >= 0; --l) {
        const bf16* in = l == 0 ? n->in0 : n->act[l - 1];
        const int cin_g = l == 0 ? 16 : 32;
        wgrad(n, l, in, cin_g, dout, dout_g, B, H, W, st);
        if (l == 0) break;
        // input gradient: forward conv of dout with the flipped transpose, masked by ReLU'(act[l-1])
        ConvArgs a{};
        a.in = dout; a.cin_g = dout_g; a.w = n->bw + n->L.bw_off[l]; a.bias = nullptr;
        bf16* o = bufs[l & 1];
        a.out = o; a.out_f = nullptr; a.cout_g = 32; a.n_out = 32; a.mask = n->act[l - 1]; a.relu = 0; a.H = H; a.W = W;
        const int cout_b = n->L.cout_pad[l] < 16 ? 16 : n->L.cout_pad[l];
        conv(cout_b, n->L.cin_pad[l] / 8, a, B, st);
        dout = o;
        dout_g = 32;
    }
}

}  // namespace

extern "C" {

size_t voldor_net_num_params(int T)
{
    if (T < 1 || T > 8) return 0;
    return net_layout(T).n_params;
}

voldor_status voldor_net_create(int T, voldor_net** out)
{
    if (!out) return VOLDOR_ERR_INVALID_ARG;
    *out = nullptr;
    if (T < 1 || T > 8) return VOLDOR_ERR_INVALID_ARG;
    voldor_net* n = new (std::nothrow) voldor_net();
    if (!n) return VOLDOR_ERR_OOM;
    n->T = T;
    n->L = net_layout(T);
    const size_t P = n->L.n_params;
    bool ok = net_ok(cudaMalloc(&n->master, P * 4)) && net_ok(cudaMalloc(&n->m, P * 4)) && net_ok(cudaMalloc(&n->v, P * 4)) &&
              net_ok(cudaMalloc(&n->grad, P * 4)) && net_ok(cudaMalloc(&n->fw, n->L.n_fw * sizeof(bf16))) &&
              net_ok(cudaMalloc(&n->bw, n->L.n_bw * sizeof(bf16))) && net_ok(cudaMalloc(&n->fbias, kNetLayers * kNetWidth * 4)) &&
              net_ok(cudaMalloc(&n->loss, 4)) && net_ok(cudaMalloc(&n->align, 8 * sizeof(float))) &&
              net_ok(cudaMalloc(&n->hist, 2 * kAlignBins * sizeof(unsigned)));
    if (ok) ok = net_ok(cudaMemset(n->master, 0, P * 4)) && net_ok(cudaMemset(n->m, 0, P * 4)) &&
                 net_ok(cudaMemset(n->v, 0, P * 4)) && net_ok(cudaMemset(n->grad, 0, P * 4));
    if (!ok) {
        cudaGetLastError();
        voldor_net_destroy(n);
        return VOLDOR_ERR_OOM;
    }
    *out = n;
    return VOLDOR_OK;
}

void voldor_net_destroy(voldor_net* n)
{
    if (!n) return;
    cudaDeviceSynchronize();
    net_free_acts(n);
    cudaFree(n->master); cudaFree(n->m); cudaFree(n->v); cudaFree(n->grad);
    cudaFree(n->fw); cudaFree(n->bw); cudaFree(n->fbias); cudaFree(n->loss);
    cudaFree(n->align); cudaFree(n->hist); cudaFree(n->fsum);
    cudaGetLastError();
    delete n;
}

voldor_status voldor_net_set_weights(voldor_net* n, const float* host, size_t count)
{
    if (!n || !host || count != n->L.n_params) return VOLDOR_ERR_INVALID_ARG;
    for (size_t i = 0; i < count; ++i)
        if (!std::isfinite(host[i])) return VOLDOR_ERR_INVALID_ARG;
    if (!net_ok(cudaMemcpy(n->master, host, count * 4, cudaMemcpyHostToDevice))) return VOLDOR_ERR_CUDA;
    cudaMemset(n->m, 0, count * 4);
    cudaMemset(n->v, 0, count * 4);
    n->step = 0;
    pack(n, nullptr);
    return net_ok(cudaDeviceSynchronize()) ? VOLDOR_OK : VOLDOR_ERR_CUDA;
}

voldor_status voldor_net_get_weights(voldor_net* n, float* host, size_t count)
{
    if (!n || !host || count != n->L.n_params) return VOLDOR_ERR_INVALID_ARG;
    return net_ok(cudaMemcpy(host, n->master, count * 4, cudaMemcpyDeviceToHost)) ? VOLDOR_OK : VOLDOR_ERR_CUDA;
}

voldor_status voldor_net_get_grads(voldor_net* n, float* host, size_t count)
{
    if (!n || !host || count != n->L.n_params) return VOLDOR_ERR_INVALID_ARG;
    return net_ok(cudaMemcpy(host, n->grad, count * 4, cudaMemcpyDeviceToHost)) ? VOLDOR_OK : VOLDOR_ERR_CUDA;
}

voldor_status voldor_net_forward(voldor_net* n, const void* flows, int flow_dtype, int B, int H, int W, float* pred,
                                 void* stream)
{
    if (!n || !flows || !pred || B < 1 || H < 1 || W < 1 || (size_t)B * n->T > 65535) return VOLDOR_ERR_INVALID_ARG;
    if (flow_dtype != VOLDOR_FLOW_F32 && flow_dtype != VOLDOR_FLOW_F16) return VOLDOR_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    voldor_status s = net_reserve(n, (size_t)B * H * W, (size_t)B * n->T);
    if (s != VOLDOR_OK) return s;
    forward(n, flows, flow_dtype == VOLDOR_FLOW_F16, B, H, W, st);
    if (!net_ok(cudaMemcpyAsync(pred, n->pred, (size_t)B * H * W * 8 * sizeof(float), cudaMemcpyDeviceToDevice, st)))
        return VOLDOR_ERR_CUDA;
    return net_ok(cudaGetLastError()) ? VOLDOR_OK : VOLDOR_ERR_CUDA;
}

voldor_status voldor_net_train_step(voldor_net* n, const void* flows, int flow_dtype, const float* target, int B, int H,
                                    int W, float lr, float lam_r, float* loss_host, void* stream)
{
    if (!n || !flows || !target || B < 1 || H < 1 || W < 1 || (size_t)B * n->T > 65535 || !(lr >= 0.f))
        return VOLDOR_ERR_INVALID_ARG;
    if (flow_dtype != VOLDOR_FLOW_F32 && flow_dtype != VOLDOR_FLOW_F16) return VOLDOR_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    voldor_status s = net_reserve(n, (size_t)B * H * W, (size_t)B * n->T);
    if (s != VOLDOR_OK) return s;
    forward(n, flows, flow_dtype == VOLDOR_FLOW_F16, B, H, W, st);
    backward(n, target, B, H, W, lam_r, st);
    if (lr > 0.f) {
        n->step += 1;
        const float b1 = 0.9f, b2 = 0.999f;
        const float c1 = 1.f - powf(b1, (float)n->step), c2 = 1.f - powf(b2, (float)n->step);
        const size_t P = n->L.n_params;
        k_adam<<<(unsigned)((P + 255) / 256), 256, 0, st>>>(n->master, n->m, n->v, n->grad, P, lr, b1, b2, 1e-8f, c1, c2);
        pack(n, st);
    }
    if (loss_host && !net_ok(cudaMemcpyAsync(loss_host, n->loss, 4, cudaMemcpyDeviceToHost, st))) return VOLDOR_ERR_CUDA;
    if (!net_ok(cudaStreamSynchronize(st))) return VOLDOR_ERR_CUDA;
    return net_ok(cudaGetLastError()) ? VOLDOR_OK : VOLDOR_ERR_CUDA;
}

}  // extern "C"

// The learned bootstrap: forward pass on the window's flows, theta and W from
// the prediction; called by voldor_bootstrap_learned.
namespace vd {
voldor_status net_bootstrap(voldor_net* n, const void* flows, int f16, int W, int H, int T, float d_min, float d_max,
                            int flags, float* theta, float* wmap, cudaStream_t st, int* kernels)
{
    *kernels = 0;
    if (!n || n->T != T) return VOLDOR_ERR_INVALID_ARG;
    if (!flags) return VOLDOR_OK;
    voldor_status s = net_reserve(n, (size_t)W * H, (size_t)T);
    if (s != VOLDOR_OK) return s;
    forward(n, flows, f16, 1, H, W, st);
    const int N = W * H;
    const unsigned nb = (unsigned)std::min(152 * 2, (N + 255) / 256);
    *kernels = 8 + 1;
    const bool depth = flags & VOLDOR_LEARNED_DEPTH;
    if (depth) {
        cudaMemsetAsync(n->hist, 0, 2 * kAlignBins * sizeof(unsigned), st);
        for (int level = 0; level < 2; ++level) {
            k_align_hist<<<nb, 256, 0, st>>>(n->pred, 8, theta, N, d_min, d_max, n->align, level, n->hist);
            k_align_select<<<1, 32, 0, st>>>(n->hist, level, n->align);
        }
        *kernels += 4;
    }
    k_net_to_state<<<(N + 255) / 256, 256, 0, st>>>(n->pred, 8, N, T, d_min, d_max, n->align,
                                                    depth ? theta : nullptr,
                                                    (flags & VOLDOR_LEARNED_RIGIDNESS) ? wmap : nullptr);
    return net_ok(cudaGetLastError()) ? VOLDOR_OK : VOLDOR_ERR_CUDA;
}
}  // namespace vd
