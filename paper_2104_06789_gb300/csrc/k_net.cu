// Learned depth / rigidness proposal: a 6-layer 3x3 convolutional network
// (2T -> 32 -> 32 -> 32 -> 32 -> 32 -> 2, ReLU between layers) that reads the
// flow stack of a window and predicts, per pixel of I_0, a log-depth and a
// rigidness logit used in place of the triangulation bootstrap. BF16
// activations and weights, FP32 accumulation: the convolutions of the forward
// pass and of the input gradient on tcgen05 (TMEM accumulators, TMA row
// loads), the weight gradient on tcgen05 too (operands transposed into
// shared memory with ldmatrix / stmatrix); FP32 Adam on master weights.
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
#include <mutex>
#include <new>
#include <vector>

#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include "voldor_internal.cuh"

namespace vd {

typedef __nv_bfloat16 bf16;

constexpr int kNetLayers = 6;
constexpr int kNetWidth = 32;
constexpr int kAlignBins = 2048;                // histogram bins per level of the median search
constexpr float kAlignRange = 16.f;             // first level covers log-ratios in [-16, 16)

__device__ __forceinline__ uint32_t smem_addr(const void* p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void ldsm_x4_t(uint32_t addr, uint32_t& r0, uint32_t& r1, uint32_t& r2, uint32_t& r3)
{
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3) : "r"(addr));
}

// ---------------------------------------------------------------------------
// 3x3 convolution on the fifth-generation tensor cores (implicit GEMM):
// out[p][n] = sum_{tap, c} in[p + off(tap)][c] w[n][tap][c] (+ bias[n]).
//
// A CTA owns a strip of kTcM = 128 output pixels of a row and walks down
// kTcRows rows of it (persistent over strips). Warp roles:
//   warp 4, one lane: TMA loads of input rows (box 8 channels x 130 columns,
//     zero fill outside the image) into a ring of kTcSlots row slots laid out
//     [channel block][column][8 channels], which is the K-major, unswizzled
//     core-matrix layout of the A operand: an A tile of 128 pixels x 16
//     channels is a descriptor into the slot (8-pixel groups 128 B apart,
//     the two 8-channel halves one channel-block row apart), and the taps'
//     column shift kx is 16 kx bytes on its start address.
//   warp 5, one lane: per output row, 9 taps x CIN/16 tcgen05.mma
//     (M = 128, N, K = 16, BF16 in, FP32 accumulators in TMEM), cycling
//     through kTcAcc accumulators, committed to mbarriers that release the
//     accumulator to the epilogue and the oldest input row to the loader.
//   warps 0-3: epilogue: tcgen05.ld of the accumulator rows of their 32 TMEM
//     lanes (one pixel per thread), bias, ReLU, the ReLU mask of a previous
//     activation (input gradient), bf16 or fp32 stores.
// Weights [N][9][CIN] are staged once per CTA in the B operand's core-matrix
// layout. Every mbarrier wait is bounded: on expiry the CTA raises *err,
// drains its own copies and MMAs, frees its TMEM and returns.
// ---------------------------------------------------------------------------
struct ConvArgs {
    const bf16* in;
    int cin_g;
    const bf16* w;          // [w_rows][9][CIN] bf16; rows w_rows..N-1 are taken as zero
    int w_rows;
    const float* bias;      // N or null
    bf16* out;              // bf16 output (channel stride cout_g) or null
    float* out_f;           // fp32 output (channel stride cout_g) or null
    int cout_g;
    int n_out;              // real output channels written
    const bf16* mask;       // zero the output where mask <= 0 (channel stride cout_g), or null
    int relu;
    int H, W, B;
    int* err;               // set to 1 if a wait expired
};

constexpr int kTcM = 128;                        // output pixels per row strip (MMA M)
constexpr int kTcCols = kTcM + 2;                // input columns per row slot
constexpr int kTcRowBytes = 2176;                // one channel block of a slot: 130 x 16 B, padded to 128 B
constexpr int kTcSlots = 6;                      // input-row ring slots
constexpr int kTcAcc = 8;                        // TMEM accumulator slots (output rows in flight)
constexpr int kTcCtasPerSm = 2;
constexpr int kTcRows = 16;                      // output rows per work item
constexpr int kTcThreads = 192;
constexpr long long kTcWaitLimit = 1ll << 24;    // polls of one mbarrier phase before giving up

template <int CIN, int N>
struct TcShape {
    static constexpr int kCB = CIN / 8;                          // channel blocks
    static constexpr int kSlotBytes = kCB * kTcRowBytes;
    static constexpr int kSlotTxBytes = kCB * kTcCols * 16;         // bytes the row's TMA boxes deliver
    static constexpr int kKSteps = 3 * CIN / 16;                 // K steps per input row (kx, channel pairs)
    static constexpr int kWStepBytes = 3 * N * 16 * 2;           // one K step of B: the three ky blocks
    static constexpr int kRingBytes = kTcSlots * kSlotBytes;
    static constexpr int kWBytes = kKSteps * kWStepBytes;
    // ring | weights | barriers: full[slots] empty[slots] acc_full[acc] acc_empty[acc] done |
    // tmem address | abort flag
    static constexpr int kBarOff = kRingBytes + kWBytes;
    static constexpr int kBarBytes = ((2 * kTcSlots + 2 * kTcAcc + 1) * 8 + 15) / 16 * 16;
    static constexpr int kSmemBytes = kBarOff + kBarBytes + 16;
    static constexpr int kTmemCols = kTcAcc * N <= 32 ? 32 : (kTcAcc * N <= 64 ? 64 : (kTcAcc * N <= 128 ? 128 : 256));
};

// Instruction descriptor of an M = 128, N = n, BF16 x BF16 -> FP32 MMA, both operands K-major.
__host__ __device__ constexpr uint32_t tc_idesc(int n)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(kTcM >> 4) << 24);
}

__device__ __forceinline__ void tc_mbar_init(uint32_t bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count));
}

__device__ __forceinline__ bool tc_try_wait(uint32_t bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile("{\n .reg .pred P;\n mbarrier.try_wait.parity.shared::cta.b64 P, [%1], %2;\n selp.u32 %0, 1, 0, P;\n}"
                 : "=r"(ok) : "r"(bar), "r"(parity) : "memory");
    return ok != 0;
}

// Bounded wait; false (and *bad set) on expiry or when another role already gave up.
__device__ __forceinline__ bool tc_wait(uint32_t bar, uint32_t parity, volatile int* bad)
{
    for (long long i = 0; i < kTcWaitLimit; ++i) {
        if (tc_try_wait(bar, parity)) return true;
        if ((i & 1023) == 1023 && *bad) return false;
    }
    *bad = 1;
    return false;
}

__device__ __forceinline__ void tc_arrive(uint32_t bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void tc_expect_tx(uint32_t bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ void tc_tma_row(uint32_t dst, const CUtensorMap* map, int c, int x, int y, int b, uint32_t bar)
{
    asm volatile("cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], [%6];"
                 ::"r"(dst), "l"(reinterpret_cast<uint64_t>(map)), "r"(c), "r"(x), "r"(y), "r"(b), "r"(bar) : "memory");
}

// Shared-memory matrix descriptor, K-major without swizzle: start, leading
// (K-direction core-matrix) offset, stride (M/N-direction 8-row group) offset.
__device__ __forceinline__ uint64_t tc_desc(uint32_t addr, uint32_t lbo, uint32_t sbo)
{
    return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

__device__ __forceinline__ void tc_mma(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc)
{
    asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                 " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}"
                 ::"r"(d_tmem), "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void tc_commit(uint32_t bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

template <int NC>
__device__ __forceinline__ void tc_ld(uint32_t taddr, float* v);

template <>
__device__ __forceinline__ void tc_ld<32>(uint32_t taddr, float* v)
{
    uint32_t r[32];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
                 "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                   "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
                   "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
                   "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
                 : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

template <>
__device__ __forceinline__ void tc_ld<16>(uint32_t taddr, float* v)
{
    uint32_t r[16];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                   "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
                 : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// Work item i: image b, strip sx (128 columns), row chunk cy (kTcRows rows).
struct TcItem {
    int b, x0, y0, rows;
};

__device__ __forceinline__ TcItem tc_item(int i, int H, int W)
{
    const int strips = (W + kTcM - 1) / kTcM, chunks = (H + kTcRows - 1) / kTcRows;
    TcItem t;
    t.b = i / (strips * chunks);
    const int r = i % (strips * chunks);
    t.x0 = (r % strips) * kTcM;
    t.y0 = (r / strips) * kTcRows;
    t.rows = min(kTcRows, H - t.y0);
    return t;
}

// Zero 8 * X consecutive TMEM columns of the warp's 32 lanes.
template <int X>
__device__ __forceinline__ void tc_zero(uint32_t taddr)
{
    const uint32_t z = 0u;
#pragma unroll
    for (int i = 0; i < X; ++i)
        asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1,%1,%1,%1,%1,%1,%1,%1};" ::"r"(taddr + 8 * i), "r"(z)
                     : "memory");
}

template <int CIN, int N>
__global__ void __launch_bounds__(kTcThreads, kTcCtasPerSm) k_conv_tc(const __grid_constant__ CUtensorMap tin, ConvArgs a)
{
    using S = TcShape<CIN, N>;
    extern __shared__ __align__(1024) unsigned char smem[];
    const uint32_t sbase = smem_addr(smem);
    const uint32_t ring = sbase, wsm = sbase + S::kRingBytes, bars = sbase + S::kBarOff;
    const uint32_t full = bars, empty = bars + kTcSlots * 8, acc_full = bars + 2 * kTcSlots * 8,
                   acc_empty = acc_full + kTcAcc * 8, done = acc_empty + kTcAcc * 8;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + S::kBarOff + S::kBarBytes);
    volatile int& bad = *reinterpret_cast<volatile int*>(smem + S::kBarOff + S::kBarBytes + 4);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int n_items = a.B * ((a.H + kTcRows - 1) / kTcRows) * ((a.W + kTcM - 1) / kTcM);

    // weights -> B operand layout: [K step][n group][k half][8 rows][8 channels] with
    // K step s = kx * (CIN / 16) + cp and n = blk * N + co, blk = 2 - ky
    for (int i = threadIdx.x; i < S::kKSteps * 3 * N * 2; i += blockDim.x) {
        const int st = i / (3 * N * 2), rem = i % (3 * N * 2);
        const int n = rem >> 1, kh = rem & 1;
        const int kx = st / (CIN / 16), cp = st % (CIN / 16);
        const int co = n % N, ky = 2 - n / N;
        uint4 v = make_uint4(0, 0, 0, 0);
        if (co < a.w_rows) v = *reinterpret_cast<const uint4*>(a.w + ((size_t)co * 9 + ky * 3 + kx) * CIN + cp * 16 + kh * 8);
        *reinterpret_cast<uint4*>(smem + S::kRingBytes + st * S::kWStepBytes + (n >> 3) * 256 + kh * 128 + (n & 7) * 16) = v;
    }
    if (threadIdx.x == 0) {
        for (int i = 0; i < kTcSlots; ++i) {
            tc_mbar_init(full + 8 * i, 1);
            tc_mbar_init(empty + 8 * i, 1);
        }
        for (int i = 0; i < kTcAcc; ++i) {
            tc_mbar_init(acc_full + 8 * i, 1);
            tc_mbar_init(acc_empty + 8 * i, 4 * 32);
        }
        tc_mbar_init(done, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        bad = 0;
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(tmem_slot)),
                     "r"((uint32_t)S::kTmemCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");     // weights visible to the tensor cores
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;
    if (warp < 4) {                                   // every accumulator slot starts at zero
        tc_zero<kTcAcc * N / 8>(tmem + ((uint32_t)(warp * 32) << 16));
        asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");

    if (warp == 4) {
        if (lane == 0) {
            // loader
            uint32_t ld = 0;
            for (int it = blockIdx.x; it < n_items && !bad; it += gridDim.x) {
                const TcItem t = tc_item(it, a.H, a.W);
                for (int r = t.y0 - 1; r <= t.y0 + t.rows && !bad; ++r, ++ld) {
                    const uint32_t slot = ld % kTcSlots;
                    if (ld >= kTcSlots && !tc_wait(empty + 8 * slot, ((ld / kTcSlots) - 1) & 1, &bad)) break;
                    tc_expect_tx(full + 8 * slot, (uint32_t)S::kSlotTxBytes);
                    for (int cb = 0; cb < S::kCB; ++cb)
                        tc_tma_row(ring + slot * S::kSlotBytes + cb * kTcRowBytes, &tin, cb * 8, t.x0 - 1, r, t.b,
                                   full + 8 * slot);
                }
            }
            // the last loads may still be landing when another role gave up
            for (uint32_t j = ld > kTcSlots ? ld - kTcSlots : 0; j < ld; ++j) {
                for (long long i = 0; i < kTcWaitLimit; ++i)
                    if (tc_try_wait(full + 8 * (j % kTcSlots), (j / kTcSlots) & 1)) break;
            }
        }
    } else if (warp == 5) {
        if (lane == 0) {
            // MMA issuer: tick k of an item consumes input row y0 - 1 + k (all three
            // kx shifts, N = 3 N columns: ky = 2, 1, 0 for output rows k - 2, k - 1,
            // k of the item), so output row j accumulates ky = 0, 1, 2 over ticks
            // j, j + 1, j + 2; output row g of the CTA's work sits in TMEM slot
            // g % kTcAcc, zeroed by the epilogue after it reads it out
            uint32_t ld = 0, G = 0;
            for (int it = blockIdx.x; it < n_items && !bad; it += gridDim.x) {
                const TcItem t = tc_item(it, a.H, a.W);
                for (int k = 0; k < t.rows + 2; ++k, ++ld) {
                    const uint32_t slot = ld % kTcSlots;
                    if (!tc_wait(full + 8 * slot, (ld / kTcSlots) & 1, &bad)) break;
                    const int b0 = max(0, 2 - k), b1 = min(3, t.rows - k + 2);
                    if (b1 == 3) {                               // first contribution to row k
                        const uint32_t gn = G + k;
                        if (gn >= kTcAcc && !tc_wait(acc_empty + 8 * (gn % kTcAcc), ((gn / kTcAcc) - 1) & 1, &bad)) break;
                    }
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    const uint32_t g0 = G + k - 2 + b0;
                    const int s0 = g0 % kTcAcc, nb = b1 - b0, nb1 = min(nb, kTcAcc - s0);
                    const uint32_t d1 = tmem + s0 * N, i1 = tc_idesc(nb1 * N), i2 = tc_idesc((nb - nb1) * N);
                    const uint32_t row = ring + slot * S::kSlotBytes;
#pragma unroll
                    for (int kx = 0; kx < 3; ++kx)
#pragma unroll
                        for (int cp = 0; cp < CIN / 16; ++cp) {
                            const int st = kx * (CIN / 16) + cp;
                            const uint64_t ad = tc_desc(row + cp * 2 * kTcRowBytes + kx * 16, kTcRowBytes, 128);
                            const uint32_t bb = wsm + st * S::kWStepBytes + b0 * N * 32;
                            tc_mma(d1, ad, tc_desc(bb, 128, 256), i1, 1u);
                            if (nb1 < nb) tc_mma(tmem, ad, tc_desc(bb + nb1 * N * 32, 128, 256), i2, 1u);
                        }
                    tc_commit(empty + 8 * slot);                 // the input row is free once these are done
                    if (b0 == 0) tc_commit(acc_full + 8 * ((G + k - 2) % kTcAcc));   // row k - 2 complete
                }
                if (bad) break;
                G += t.rows;
            }
            tc_commit(done);                  // arrives once every MMA issued above has completed
            for (long long i = 0; i < kTcWaitLimit; ++i)
                if (tc_try_wait(done, 0)) break;
        }
    } else {
        // epilogue: warp w reads TMEM lanes 32w .. 32w + 31 = pixels x0 + 32w + lane
        float bias[N];
#pragma unroll
        for (int n = 0; n < N; ++n) bias[n] = a.bias ? __ldg(a.bias + n) : 0.f;
        uint32_t g = 0;
        bool go = true;
        for (int it = blockIdx.x; it < n_items && go; it += gridDim.x) {
            const TcItem t = tc_item(it, a.H, a.W);
            for (int k = 0; k < t.rows; ++k, ++g) {
                const uint32_t buf = g % kTcAcc;
                // every lane polls; the warp proceeds only together (tcgen05.ld is warp-wide)
                go = __all_sync(0xffffffffu, tc_wait(acc_full + 8 * buf, (g / kTcAcc) & 1, &bad));
                if (!go) break;
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                float v[N];
                const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + buf * N;
                tc_ld<N>(taddr, v);
                tc_zero<N / 8>(taddr);
                asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
                asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                tc_arrive(acc_empty + 8 * buf);
                const int px = t.x0 + warp * 32 + lane, py = t.y0 + k;
                if (px >= a.W) continue;
                const size_t o = (((size_t)t.b * a.H + py) * a.W + px) * a.cout_g;
#pragma unroll
                for (int n = 0; n < N; ++n) v[n] += bias[n];
                if (a.relu) {
#pragma unroll
                    for (int n = 0; n < N; ++n) v[n] = fmaxf(v[n], 0.f);
                }
                if (a.mask) {
#pragma unroll
                    for (int q = 0; q < N / 8; ++q) {
                        const uint4 m = *reinterpret_cast<const uint4*>(a.mask + o + 8 * q);
                        const bf16* mb = reinterpret_cast<const bf16*>(&m);
#pragma unroll
                        for (int e = 0; e < 8; ++e)
                            if (!(__bfloat162float(mb[e]) > 0.f)) v[8 * q + e] = 0.f;
                    }
                }
                if (a.out) {
#pragma unroll
                    for (int q = 0; q < N / 8; ++q) {
                        if (8 * q >= a.n_out) break;
                        __align__(16) bf16 h[8];
#pragma unroll
                        for (int e = 0; e < 8; ++e) h[e] = __float2bfloat16_rn(v[8 * q + e]);
                        *reinterpret_cast<uint4*>(a.out + o + 8 * q) = *reinterpret_cast<const uint4*>(h);
                    }
                }
                if (a.out_f) {
#pragma unroll
                    for (int q = 0; q < N / 4; ++q) {
                        if (4 * q >= a.n_out) break;
                        *reinterpret_cast<float4*>(a.out_f + o + 4 * q) =
                            make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
                    }
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"((uint32_t)S::kTmemCols));
    }
    if (threadIdx.x == 0 && bad) atomicExch(a.err, 1);
}

// cuTensorMapEncodeTiled through the runtime's driver entry point (no link
// against the driver library).
static PFN_cuTensorMapEncodeTiled_v12000 g_encode_tiled = nullptr;
static std::once_flag g_encode_once;

static bool tensor_map_rows(CUtensorMap* m, const bf16* base, int C, int W, int H, int B)
{
    std::call_once(g_encode_once, [] {
        void* fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess && fn)
            g_encode_tiled = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    });
    if (!g_encode_tiled) return false;
    const cuuint64_t dims[4] = {(cuuint64_t)C, (cuuint64_t)W, (cuuint64_t)H, (cuuint64_t)B};
    const cuuint64_t strides[3] = {(cuuint64_t)C * 2, (cuuint64_t)W * C * 2, (cuuint64_t)H * W * C * 2};
    const cuuint32_t box[4] = {8, (cuuint32_t)kTcCols, 1, 1};
    const cuuint32_t es[4] = {1, 1, 1, 1};
    return g_encode_tiled(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<bf16*>(base), dims, strides, box, es,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Per-device launch state: SM count, and whether an instance's dynamic
// shared-memory limit has been raised on that device.
constexpr int kTcMaxDevices = 64;
static std::mutex g_tc_mutex;
static int g_tc_sms[kTcMaxDevices];

template <int CIN, int N>
static bool launch_conv_tc(const ConvArgs& a, cudaStream_t st)
{
    using S = TcShape<CIN, N>;
    static bool attr[kTcMaxDevices];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kTcMaxDevices) return false;
    int sms = 0;
    {
        std::lock_guard<std::mutex> lock(g_tc_mutex);
        if (!attr[dev]) {
            if (cudaFuncSetAttribute(k_conv_tc<CIN, N>, cudaFuncAttributeMaxDynamicSharedMemorySize, S::kSmemBytes) !=
                cudaSuccess)
                return false;
            attr[dev] = true;
        }
        if (g_tc_sms[dev] <= 0 &&
            (cudaDeviceGetAttribute(&g_tc_sms[dev], cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
             g_tc_sms[dev] <= 0))
            g_tc_sms[dev] = 152;
        sms = g_tc_sms[dev];
    }
    CUtensorMap m;
    if (!tensor_map_rows(&m, a.in, CIN, a.W, a.H, a.B)) return false;
    const int items = a.B * ((a.H + kTcRows - 1) / kTcRows) * ((a.W + kTcM - 1) / kTcM);
    const int grid = std::min(items, kTcCtasPerSm * sms);
    k_conv_tc<CIN, N><<<grid, kTcThreads, S::kSmemBytes, st>>>(m, a);
    return true;
}

// Arguments of the weight-gradient kernel below.
struct WgradArgs {
    const bf16* in;
    int cin_g;
    const bf16* dout;       // channel stride cout_g
    int cout_g;
    float* dw;              // [n_out][9][cin_real]
    float* db;              // [n_out]
    float* part;            // [gridDim.x][9 CIN + 1][NCO] each CTA's sums
    float* part2;           // [ceil(gridDim.x / kWgGroup)][9 CIN + 1][NCO] their group sums
    int n_out, cin_real;
    int H, W, B;
    int* err;               // set to 1 if a bounded wait expired
};

// ---------------------------------------------------------------------------
// Weight gradient on the fifth-generation tensor cores:
// dw[co][tap][ci] += sum_p dout[p][co] in[p + off(tap)][ci] and
// db[co] += sum_p dout[p][co], as one GEMM per layer: D[m][n] =
// sum_k A[m][k] B[n][k] with
// m = tap * CIN + ci (the 9 CIN rows of the layer's input, shifted by the
// tap), n = output channel, k = pixel; one extra row of ones (m = 9 CIN)
// gives the bias gradient sum_p dout[p][n]. Rows are cut into 128-row M tiles
// (tcgen05.mma M = 128, N = NCO, K = 16, BF16 in, FP32 accumulators in TMEM
// that persist over all of a CTA's work items).
//
// A work item is KP = 64 consecutive output pixels of one image row. Its
// three input rows (66 pixels each, zero outside the image) and its output
// gradients are staged pixel-major in shared memory, then transposed 8 x 8 at
// a time (ldmatrix .trans, then stmatrix) into the K-major, unswizzled
// core-matrix layout of the two operands: element (m, k) of an M tile at
// (k / 8) * 2048 + (m / 8) * 128 + (m % 8) * 16 + (k % 8) * 2 bytes, and
// (n, k) of B at (k / 8) * (NCO / 8) * 128 + (n / 8) * 128 + (n % 8) * 16 +
// (k % 8) * 2. One thread issues the item's MMAs and commits them to an
// mbarrier; the next item's pixel-major staging overlaps them, and every
// thread waits on the commit (bounded) before overwriting the operands. At
// the end each thread reads its TMEM row (tcgen05.ld) and adds it to the
// FP32 gradients with atomics.
// ---------------------------------------------------------------------------
constexpr int kWgKP = 64;                                 // pixels per work item (K)
constexpr int kWgThreads = 128;
constexpr int kWgCtasPerSm = 3;                          // weight-gradient grid: at most this many CTAs per SM
constexpr int kWgPartRows = 9 * 32 + 1;                   // largest per-CTA partial: rows x 32 columns

template <int CIN, int NCO>
struct WgShape {
    static constexpr int kRows = 9 * CIN + 1;                           // + the ones row
    static constexpr int kMT = (kRows + 127) / 128;
    static constexpr int kInRowBytes = (kWgKP + 2) * CIN * 2;
    static constexpr int kInBytes = 3 * kInRowBytes;
    static constexpr int kDoBytes = kWgKP * NCO * 2;
    static constexpr int kATileBytes = (kWgKP / 8) * 2048;
    static constexpr int kBLbo = (NCO / 8) * 128;
    static constexpr int kBBytes = (kWgKP / 8) * kBLbo;
    static constexpr int kInOff = 0;
    static constexpr int kDoOff = kInOff + kInBytes;
    static constexpr int kAOff = (kDoOff + kDoBytes + 1023) / 1024 * 1024;
    static constexpr int kBOff = kAOff + kMT * kATileBytes;
    static constexpr int kBarOff = kBOff + kBBytes;
    static constexpr int kSmemBytes = kBarOff + 32;
    static constexpr int kTmemCols = kMT * NCO <= 32 ? 32 : (kMT * NCO <= 64 ? 64 : 128);
    static constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(NCO >> 3) << 17) |
                                       ((uint32_t)(128 >> 4) << 24);
};

__device__ __forceinline__ void stsm_x4(uint32_t addr, uint32_t r0, uint32_t r1, uint32_t r2, uint32_t r3)
{
    asm volatile("stmatrix.sync.aligned.m8n8.x4.shared.b16 [%0], {%1, %2, %3, %4};" ::"r"(addr), "r"(r0), "r"(r1),
                 "r"(r2), "r"(r3) : "memory");
}

template <int CIN, int NCO>
__global__ void __launch_bounds__(kWgThreads) k_wgrad_tc(const __grid_constant__ WgradArgs a)
{
    using S = WgShape<CIN, NCO>;
    extern __shared__ __align__(1024) unsigned char smem[];
    const uint32_t sbase = smem_addr(smem);
    const uint32_t in_s = sbase + S::kInOff, do_s = sbase + S::kDoOff, A_s = sbase + S::kAOff, B_s = sbase + S::kBOff;
    const uint32_t bar = sbase + S::kBarOff, done = bar + 8;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + S::kBarOff + 16);
    volatile int& bad = *reinterpret_cast<volatile int*>(smem + S::kBarOff + 20);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int segs = (a.W + kWgKP - 1) / kWgKP;
    const int n_items = a.B * a.H * segs;

    // constant rows of A in every M tile: the ones row (bias gradient) and zero padding
    for (int i = tid; i < S::kMT * 128 * kWgKP; i += blockDim.x) {
        const int m = i / kWgKP, k = i % kWgKP;
        if (m < 9 * CIN) continue;
        const int mt = m / 128, mm = m % 128;
        const uint32_t off = S::kAOff + mt * S::kATileBytes + (k / 8) * 2048 + (mm / 8) * 128 + (mm % 8) * 16 + (k % 8) * 2;
        *reinterpret_cast<bf16*>(smem + off) = __float2bfloat16_rn(m == 9 * CIN ? 1.f : 0.f);
    }
    if (tid == 0) {
        tc_mbar_init(bar, 1);
        tc_mbar_init(done, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        bad = 0;
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(tmem_slot)),
                     "r"((uint32_t)S::kTmemCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;

    // an item's input rows and output gradients, loaded into registers one
    // item ahead (the loads of item i + 1 are in flight while item i is
    // transposed and multiplied) and stored pixel-major at the top of the loop
    constexpr int kInVec = 3 * (kWgKP + 2) * (CIN / 8), kDoVec = kWgKP * (NCO / 8);
    constexpr int kInPer = (kInVec + kWgThreads - 1) / kWgThreads, kDoPer = (kDoVec + kWgThreads - 1) / kWgThreads;
    uint4 pin[kInPer], pdo[kDoPer];
    auto fetch = [&](int it) {
        const int b = it / (a.H * segs), rem = it % (a.H * segs);
        const int y = rem / segs, x0 = (rem % segs) * kWgKP;
#pragma unroll
        for (int j = 0; j < kInPer; ++j) {
            const int i = tid + j * kWgThreads;
            pin[j] = make_uint4(0, 0, 0, 0);
            if (i < kInVec) {
                const int v = i % (CIN / 8), q = i / (CIN / 8);
                const int ky = q / (kWgKP + 2), xx = q % (kWgKP + 2);
                const int gy = y + ky - 1, gx = x0 + xx - 1;
                if (gy >= 0 && gy < a.H && gx >= 0 && gx < a.W)
                    pin[j] = *reinterpret_cast<const uint4*>(a.in + (((size_t)b * a.H + gy) * a.W + gx) * a.cin_g + v * 8);
            }
        }
#pragma unroll
        for (int j = 0; j < kDoPer; ++j) {
            const int i = tid + j * kWgThreads;
            pdo[j] = make_uint4(0, 0, 0, 0);
            if (i < kDoVec) {
                const int v = i % (NCO / 8), px = i / (NCO / 8), gx = x0 + px;
                if (gx < a.W && v * 8 < a.n_out) {
                    pdo[j] = *reinterpret_cast<const uint4*>(a.dout + (((size_t)b * a.H + y) * a.W + gx) * a.cout_g + v * 8);
                    if (v * 8 + 8 > a.n_out) {                // channels past n_out are zero
                        bf16* e = reinterpret_cast<bf16*>(&pdo[j]);
                        for (int c = a.n_out - v * 8; c < 8; ++c) e[c] = __float2bfloat16_rn(0.f);
                    }
                }
            }
        }
    };
    if (blockIdx.x < n_items) fetch(blockIdx.x);
    int local = 0;                                            // items of this CTA so far
    for (int it = blockIdx.x; it < n_items; it += gridDim.x, ++local) {
        // pixel-major staging of this item (the operands of the previous item
        // may still be read by its MMAs; these buffers are not)
#pragma unroll
        for (int j = 0; j < kInPer; ++j) {
            const int i = tid + j * kWgThreads;
            if (i < kInVec) {
                const int v = i % (CIN / 8), q = i / (CIN / 8);
                const int ky = q / (kWgKP + 2), xx = q % (kWgKP + 2);
                *reinterpret_cast<uint4*>(smem + S::kInOff + ky * S::kInRowBytes + xx * CIN * 2 + v * 16) = pin[j];
            }
        }
#pragma unroll
        for (int j = 0; j < kDoPer; ++j) {
            const int i = tid + j * kWgThreads;
            if (i < kDoVec) {
                const int v = i % (NCO / 8), px = i / (NCO / 8);
                *reinterpret_cast<uint4*>(smem + S::kDoOff + px * NCO * 2 + v * 16) = pdo[j];
            }
        }
        if (it + (int)gridDim.x < n_items) fetch(it + gridDim.x);
        // the previous item's MMAs have read A and B; a wait that expires sets
        // `bad`, which every thread reads after the same barrier
        if (local > 0) tc_wait(bar, (uint32_t)((local - 1) & 1), &bad);
        __syncthreads();
        if (bad) break;
        // 8 x 8 transposes into the K-major operands: A blocks (tap, ci group, k group), then B blocks
        constexpr int kABlocks = 9 * (CIN / 8) * (kWgKP / 8), kBBlocks = (NCO / 8) * (kWgKP / 8);
        static_assert((kABlocks + kBBlocks) % 16 == 0, "four x4 transposes per round, one per warp");
        for (int q0 = warp * 4; q0 < kABlocks + kBBlocks; q0 += 16) {
            const int blk = q0 + (lane >> 3), r = lane & 7;
            uint32_t src, dst;
            if (blk < kABlocks) {
                const int kg = blk % (kWgKP / 8), g = (blk / (kWgKP / 8)) % (CIN / 8), tap = blk / ((kWgKP / 8) * (CIN / 8));
                const int ky = tap / 3, kx = tap % 3;
                const int m = tap * CIN + g * 8 + r, mt = m / 128, mm = m % 128;
                src = in_s + ky * S::kInRowBytes + (8 * kg + r + kx) * CIN * 2 + g * 16;
                dst = A_s + mt * S::kATileBytes + kg * 2048 + (mm / 8) * 128 + r * 16;
            } else {
                const int bb = blk - kABlocks, kg = bb % (kWgKP / 8), g = bb / (kWgKP / 8);
                src = do_s + (8 * kg + r) * NCO * 2 + g * 16;
                dst = B_s + kg * S::kBLbo + g * 128 + r * 16;
            }
            // lane l gives row l % 8 of block l / 8: the transposing load, then the
            // plain store, writes each block's transpose to the destination rows
            uint32_t r0, r1, r2, r3;
            ldsm_x4_t(src, r0, r1, r2, r3);
            stsm_x4(dst, r0, r1, r2, r3);
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
            for (int mt = 0; mt < S::kMT; ++mt)
#pragma unroll
                for (int s16 = 0; s16 < kWgKP / 16; ++s16) {
                    const uint64_t ad = tc_desc(A_s + mt * S::kATileBytes + s16 * 2 * 2048, 2048, 128);
                    const uint64_t bd = tc_desc(B_s + s16 * 2 * S::kBLbo, S::kBLbo, 128);
                    tc_mma(tmem + mt * NCO, ad, bd, S::kIdesc, (local > 0 || s16 > 0) ? 1u : 0u);
                }
            tc_commit(bar);
        }
    }
    if (tid == 0) {
        tc_commit(done);                                      // arrives once every MMA issued has completed
        bool drained = false;
        for (long long i = 0; i < kTcWaitLimit && !drained; ++i) drained = tc_try_wait(done, 0);
        if (!drained) bad = 1;
    }
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (!bad) {
        // this CTA's sums, row m (tap * CIN + ci, then the bias row) of its partial
#pragma unroll
        for (int mt = 0; mt < S::kMT; ++mt) {
            float v[NCO];
            tc_ld<NCO>(tmem + ((uint32_t)(warp * 32) << 16) + mt * NCO, v);
            if (local == 0) {
#pragma unroll
                for (int co = 0; co < NCO; ++co) v[co] = 0.f;
            }
            const int m = mt * 128 + warp * 32 + lane;
            if (m < S::kRows) {
                float4* o = reinterpret_cast<float4*>(a.part + ((size_t)blockIdx.x * S::kRows + m) * NCO);
#pragma unroll
                for (int q = 0; q < NCO / 4; ++q) o[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"((uint32_t)S::kTmemCols));
    }
    if (tid == 0 && bad) atomicExch(a.err, 1);
}

// The layer's gradients from the CTAs' partial sums, in a fixed order (so
// that a training run is bit-reproducible, unlike with floating-point
// atomics), in two levels: k_wgrad_group sums groups of kWgGroup consecutive
// CTAs (grid.y = group), k_wgrad_reduce the groups in order and writes
// dw[co][tap][ci] (row m = tap * CIN + ci) or db[co] (m = 9 CIN). Entry
// i = m * NCO + co.
constexpr int kWgGroup = 16;

template <int CIN, int NCO>
__global__ void k_wgrad_group(const float* part, int n_cta, float* part2)
{
    constexpr int R = 9 * CIN + 1;
    const int i = blockIdx.x * blockDim.x + threadIdx.x, g = blockIdx.y;
    if (i >= R * NCO) return;
    const size_t cs = (size_t)R * NCO;
    const int c0 = g * kWgGroup, c1 = min(n_cta, c0 + kWgGroup);
    float v[kWgGroup];
#pragma unroll
    for (int u = 0; u < kWgGroup; ++u) v[u] = c0 + u < c1 ? part[(size_t)(c0 + u) * cs + i] : 0.f;
    float sum = 0.f;
#pragma unroll
    for (int u = 0; u < kWgGroup; ++u) sum += v[u];
    part2[(size_t)g * cs + i] = sum;
}

template <int CIN, int NCO>
__global__ void k_wgrad_reduce(const float* part2, int n_groups, float* dw, float* db, int n_out, int cin_real)
{
    constexpr int R = 9 * CIN + 1;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= R * NCO) return;
    const int m = i / NCO, co = i % NCO;
    if (co >= n_out) return;
    const size_t cs = (size_t)R * NCO;
    float sum = 0.f;
    for (int g = 0; g < n_groups; ++g) sum += part2[(size_t)g * cs + i];
    if (m < 9 * CIN) {
        const int tap = m / CIN, ci = m % CIN;
        if (ci < cin_real) dw[((size_t)co * 9 + tap) * cin_real + ci] = sum;
    } else {
        db[co] = sum;
    }
}

// ---------------------------------------------------------------------------
// Input packing, loss, parameter packing, Adam, proposal output.
// ---------------------------------------------------------------------------
// Sum of |flow| per (image, frame), deterministic: grid (kNormBlocks, B*T);
// each block writes its partial sum, k_flow_norm_fold adds a frame's
// partials in a fixed order.
constexpr int kNormBlocks = 64;

__device__ __forceinline__ float flow_mag(float2 f)
{
    const float m = sqrtf(f.x * f.x + f.y * f.y);
    return isfinite(m) ? m : 0.f;
}

// Partial sums of |flow| per (image, frame): grid (kNormBlocks, B*T). Eight
// independent loads in flight per thread (a plain strided loop keeps one, too
// few bytes in flight for the HBM bandwidth), added in index order.
__global__ void k_flow_norm_sum(const void* flows, int f16, size_t N, float* partial)
{
    const int bt = blockIdx.y;
    const size_t stride = (size_t)gridDim.x * blockDim.x, base = (size_t)bt * N;
    float s = 0.f;
    size_t p = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    constexpr int kU = 8;
    for (; p < N; p += kU * stride) {               // the last round predicated, not a serial tail
        float2 f[kU];
#pragma unroll
        for (int u = 0; u < kU; ++u)
            f[u] = p + u * stride < N ? load_flow(flows, f16, base + p + u * stride) : make_float2(0.f, 0.f);
#pragma unroll
        for (int u = 0; u < kU; ++u) s += flow_mag(f[u]);
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    __shared__ float ws[32];
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        float t = 0.f;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += ws[w];
        partial[(size_t)bt * kNormBlocks + blockIdx.x] = t;
    }
}

// One warp per (image, frame): the frame's |flow| sum from the kNormBlocks
// partials, stored as the scale of the network input, N / sum = 1 / mean |flow|
// (0 for a frame without motion).
__global__ void k_flow_norm_fold(const float* partial, float N, float* inv)
{
    const int bt = blockIdx.x;
    float s = partial[(size_t)bt * kNormBlocks + threadIdx.x] + partial[(size_t)bt * kNormBlocks + threadIdx.x + 32];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (threadIdx.x == 0) inv[bt] = s > 0.f ? N / s : 0.f;
}

// grid (pixel blocks, B): pixel p of image b -> 16 bf16 channels (2T scaled flows, then zeros)
__global__ void k_pack_input(const void* flows, int f16, int T, int N, const float* inv, bf16* in0)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x, b = blockIdx.y;
    if (p >= N) return;
    const int Tc = T < 8 ? T : 8;
    float2 f[8];
#pragma unroll
    for (int t = 0; t < 8; ++t)
        if (t < Tc) f[t] = load_flow(flows, f16, ((size_t)b * T + t) * N + p);
    __align__(16) bf16 v[16];
#pragma unroll
    for (int t = 0; t < 8; ++t) {
        const float sc = t < Tc ? inv[b * T + t] : 0.f;
        v[2 * t] = __float2bfloat16_rn(t < Tc ? f[t].x * sc : 0.f);
        v[2 * t + 1] = __float2bfloat16_rn(t < Tc ? f[t].y * sc : 0.f);
    }
    uint4* o = reinterpret_cast<uint4*>(in0 + ((size_t)b * N + p) * 16);
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
    int* tc_err = nullptr;           // set by a convolution whose bounded wait expired
    unsigned* hist = nullptr;        // [2][kAlignBins]
    float* fsum = nullptr;           // [cap_bt] input scale N / sum |flow| per (image, frame), then [cap_bt][kNormBlocks] partials
    size_t cap_bt = 0;
    int step = 0;
    size_t cap_pix = 0;
    bf16* in0 = nullptr;            // [pix][16]
    bf16* act[kNetLayers - 1] = {}; // [pix][32]
    float* pred = nullptr;          // [pix][8]
    bf16* g16 = nullptr;            // [pix][16] gradient at the output
    bf16 *ga = nullptr, *gb = nullptr;   // [pix][32] gradient ping-pong
    float* wpart = nullptr;         // weight-gradient partial sums: [kWgCtasPerSm * SMs][kWgPartRows][32],
                                    // then their group sums (the same layout, one entry per group of CTAs)
};

namespace {

bool net_ok(cudaError_t e) { return e == cudaSuccess; }

// SM count of the current device (the weight-gradient grid is sized by it).
int net_sms()
{
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        sms <= 0)
        return 152;
    return sms;
}

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
        if (!net_ok(cudaMalloc(&n->fsum, bt * (1 + kNormBlocks) * sizeof(float)))) {
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

// Dispatch on (input channels, output channels rounded up to 16).
bool conv(int cin_pad, int n_out_pad, const ConvArgs& a, cudaStream_t st)
{
    if (a.cin_g != cin_pad) return false;
    if (cin_pad == 16 && n_out_pad == 32) return launch_conv_tc<16, 32>(a, st);
    if (cin_pad == 32 && n_out_pad == 32) return launch_conv_tc<32, 32>(a, st);
    if (cin_pad == 32 && n_out_pad == 16) return launch_conv_tc<32, 16>(a, st);
    return false;
}

// Forward pass of B images of H x W; predictions (8 floats per pixel) in
// `out`, a 16-byte aligned device buffer, or in n->pred when out is null.
// False if a convolution could not be launched.
bool forward(voldor_net* n, const void* flows, int f16, int B, int H, int W, cudaStream_t st, float* out = nullptr)
{
    const size_t N = (size_t)H * W;
    float* partial = n->fsum + n->cap_bt;
    k_flow_norm_sum<<<dim3(kNormBlocks, B * n->T), 256, 0, st>>>(flows, f16, N, partial);
    k_flow_norm_fold<<<B * n->T, 32, 0, st>>>(partial, (float)N, n->fsum);
    k_pack_input<<<dim3((unsigned)((N + 255) / 256), B), 256, 0, st>>>(flows, f16, n->T, (int)N, n->fsum, n->in0);
    const bf16* in = n->in0;
    int cin_g = 16;
    for (int l = 0; l < kNetLayers; ++l) {
        const bool last = l == kNetLayers - 1;
        ConvArgs a{};
        a.in = in; a.cin_g = cin_g; a.w = n->fw + n->L.fw_off[l]; a.bias = n->fbias + l * kNetWidth;
        a.out = last ? nullptr : n->act[l]; a.out_f = last ? (out ? out : n->pred) : nullptr;
        a.cout_g = last ? 8 : 32; a.n_out = last ? 8 : 32; a.mask = nullptr; a.relu = last ? 0 : 1; a.H = H; a.W = W;
        a.B = B; a.w_rows = n->L.cout_pad[l]; a.err = n->tc_err;
        if (!conv(n->L.cin_pad[l], last ? 16 : 32, a, st)) return false;
        if (last) break;
        in = n->act[l];
        cin_g = 32;
    }
    return true;
}

template <int CIN, int NCO>
static bool launch_wgrad_tc(const WgradArgs& a, cudaStream_t st)
{
    using S = WgShape<CIN, NCO>;
    static bool attr[kTcMaxDevices];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kTcMaxDevices) return false;
    int sms = 0;
    {
        std::lock_guard<std::mutex> lock(g_tc_mutex);
        if (!attr[dev]) {
            if (cudaFuncSetAttribute(k_wgrad_tc<CIN, NCO>, cudaFuncAttributeMaxDynamicSharedMemorySize, S::kSmemBytes) !=
                cudaSuccess)
                return false;
            attr[dev] = true;
        }
        if (g_tc_sms[dev] <= 0 &&
            (cudaDeviceGetAttribute(&g_tc_sms[dev], cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
             g_tc_sms[dev] <= 0))
            g_tc_sms[dev] = 152;
        sms = g_tc_sms[dev];
    }
    const int items = a.B * a.H * ((a.W + kWgKP - 1) / kWgKP);
    const int grid = std::min(items, kWgCtasPerSm * sms);
    k_wgrad_tc<CIN, NCO><<<grid, kWgThreads, S::kSmemBytes, st>>>(a);
    const int n_groups = (grid + kWgGroup - 1) / kWgGroup;
    const unsigned blocks = (unsigned)((S::kRows * NCO + 255) / 256);
    k_wgrad_group<CIN, NCO><<<dim3(blocks, n_groups), 256, 0, st>>>(a.part, grid, a.part2);
    k_wgrad_reduce<CIN, NCO><<<blocks, 256, 0, st>>>(a.part2, n_groups, a.dw, a.db, a.n_out, a.cin_real);
    return true;
}

void wgrad(voldor_net* n, int l, const bf16* in, int cin_g, const bf16* dout, int cout_g, int B, int H, int W, cudaStream_t st)
{
    WgradArgs a{};
    a.in = in; a.cin_g = cin_g; a.dout = dout; a.cout_g = cout_g;
    a.dw = n->grad + n->L.w_off[l]; a.db = n->grad + n->L.b_off[l];
    a.part = n->wpart;
    a.part2 = n->wpart + (size_t)kWgCtasPerSm * net_sms() * kWgPartRows * 32;
    a.n_out = n->L.cout[l]; a.cin_real = n->L.cin[l];
    a.H = H; a.W = W; a.B = B;
    a.err = n->tc_err;
    const int cinp = n->L.cin_pad[l];
    const bool wide = n->L.cout[l] > 16;
    if (cinp == 16 && wide) launch_wgrad_tc<16, 32>(a, st);
    else if (cinp == 32 && wide) launch_wgrad_tc<32, 32>(a, st);
    else if (cinp == 32 && !wide) launch_wgrad_tc<32, 16>(a, st);
}

// Backward pass after forward(); target [pix][2] (log-depth, rigidness).
bool backward(voldor_net* n, const float* tgt, int B, int H, int W, float lam_r, cudaStream_t st)
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
        a.B = B; a.w_rows = n->L.cin_pad[l]; a.err = n->tc_err;
        const int cout_b = n->L.cout_pad[l] < 16 ? 16 : n->L.cout_pad[l];
        if (!conv(cout_b, 32, a, st)) return false;
        dout = o;
        dout_g = 32;
    }
    return true;
}

// Reads (synchronising the stream) and clears the convolutions' timeout flag.
voldor_status net_status(voldor_net* n, cudaStream_t st)
{
    int e = 0;
    if (!net_ok(cudaMemcpyAsync(&e, n->tc_err, sizeof(int), cudaMemcpyDeviceToHost, st)) ||
        !net_ok(cudaStreamSynchronize(st)))
        return VOLDOR_ERR_CUDA;
    if (e) {
        cudaMemsetAsync(n->tc_err, 0, sizeof(int), st);
        return VOLDOR_ERR_TIMEOUT;
    }
    return net_ok(cudaGetLastError()) ? VOLDOR_OK : VOLDOR_ERR_CUDA;
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
              net_ok(cudaMalloc(&n->wpart, (size_t)(kWgCtasPerSm * net_sms() + (kWgCtasPerSm * net_sms() + 15) / 16) *
                                               kWgPartRows * 32 * sizeof(float))) &&
              net_ok(cudaMalloc(&n->hist, 2 * kAlignBins * sizeof(unsigned))) && net_ok(cudaMalloc(&n->tc_err, sizeof(int)));
    if (ok) ok = net_ok(cudaMemset(n->master, 0, P * 4)) && net_ok(cudaMemset(n->m, 0, P * 4)) &&
                 net_ok(cudaMemset(n->v, 0, P * 4)) && net_ok(cudaMemset(n->grad, 0, P * 4)) &&
                 net_ok(cudaMemset(n->tc_err, 0, sizeof(int)));
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
    cudaFree(n->align); cudaFree(n->hist); cudaFree(n->fsum); cudaFree(n->tc_err); cudaFree(n->wpart);
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
    if (!n || !flows || !pred || B < 1 || H < 1 || W < 1 || (size_t)B * n->T > 65535 || (size_t)H * W > 0x7fffffff)
        return VOLDOR_ERR_INVALID_ARG;
    if (flow_dtype != VOLDOR_FLOW_F32 && flow_dtype != VOLDOR_FLOW_F16) return VOLDOR_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    voldor_status s = net_reserve(n, (size_t)B * H * W, (size_t)B * n->T);
    if (s != VOLDOR_OK) return s;
    // The last layer writes the caller's buffer directly when the epilogue's
    // 16-byte stores can reach it (memory of the current device, 16-byte
    // aligned); otherwise it writes the network's own buffer, which is then
    // copied.
    cudaPointerAttributes pa{};
    bool direct = false;
    int dev = -1;
    if (((uintptr_t)pred & 15) == 0 && cudaGetDevice(&dev) == cudaSuccess) {
        if (cudaPointerGetAttributes(&pa, pred) == cudaSuccess)
            direct = (pa.type == cudaMemoryTypeDevice || pa.type == cudaMemoryTypeManaged) && pa.device == dev;
        else
            cudaGetLastError();   // a failed attribute query is not an error of the forward pass
    }
    if (!forward(n, flows, flow_dtype == VOLDOR_FLOW_F16, B, H, W, st, direct ? pred : nullptr)) return VOLDOR_ERR_CUDA;
    if (!direct &&
        !net_ok(cudaMemcpyAsync(pred, n->pred, (size_t)B * H * W * 8 * sizeof(float), cudaMemcpyDeviceToDevice, st)))
        return VOLDOR_ERR_CUDA;
    return net_status(n, st);
}

voldor_status voldor_net_train_step(voldor_net* n, const void* flows, int flow_dtype, const float* target, int B, int H,
                                    int W, float lr, float lam_r, float* loss_host, void* stream)
{
    if (!n || !flows || !target || B < 1 || H < 1 || W < 1 || (size_t)B * n->T > 65535 || (size_t)H * W > 0x7fffffff ||
        !(lr >= 0.f))
        return VOLDOR_ERR_INVALID_ARG;
    if (flow_dtype != VOLDOR_FLOW_F32 && flow_dtype != VOLDOR_FLOW_F16) return VOLDOR_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    voldor_status s = net_reserve(n, (size_t)B * H * W, (size_t)B * n->T);
    if (s != VOLDOR_OK) return s;
    if (!forward(n, flows, flow_dtype == VOLDOR_FLOW_F16, B, H, W, st) || !backward(n, target, B, H, W, lam_r, st))
        return VOLDOR_ERR_CUDA;
    if (lr > 0.f) {
        n->step += 1;
        const float b1 = 0.9f, b2 = 0.999f;
        const float c1 = 1.f - powf(b1, (float)n->step), c2 = 1.f - powf(b2, (float)n->step);
        const size_t P = n->L.n_params;
        k_adam<<<(unsigned)((P + 255) / 256), 256, 0, st>>>(n->master, n->m, n->v, n->grad, P, lr, b1, b2, 1e-8f, c1, c2);
        pack(n, st);
    }
    if (loss_host && !net_ok(cudaMemcpyAsync(loss_host, n->loss, 4, cudaMemcpyDeviceToHost, st))) return VOLDOR_ERR_CUDA;
    return net_status(n, st);
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
    if (!forward(n, flows, f16, 1, H, W, st)) return VOLDOR_ERR_CUDA;
    const int N = W * H;
    const unsigned nb = (unsigned)std::min(152 * 2, (N + 255) / 256);
    *kernels = 9 + 1;            // forward (norm sum, fold, packing, 6 convolutions), to_state
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
    return net_status(n, st);
}
}  // namespace vd
