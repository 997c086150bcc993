// Epipolar bootstrap of T_1 (Sec. 5.3 and Table 1: T_1 from the epipolar
// geometry of X_1 with a least-median-of-squares estimator).
//
//  1. k_epi_records: per pixel, the calibrated correspondence of X_1 as
//     {m0x, m0y, u/fx, v/fy} (FP32), m0 = K^-1 [x y 1]; NaN marks a pixel whose
//     flow target leaves I_1 (tested in FP64).
//  2. k_epi_samples: one thread per minimal sample: 8 Philox-drawn pixels,
//     the 8-point essential matrix (null vector of the 8 x 9 system by Gaussian
//     elimination with complete pivoting, FP64), its projection onto the
//     essential matrices (eigen-decomposition of E^T E by Jacobi rotations),
//     and a scoring form: the decomposition [t]x R with the smaller rotation,
//     as Q = R - I and unit t in FP32.
//  3. k_epi_hist / k_epi_select, three passes: the exact lower median of every
//     sample's Sampson errors over all valid pixels by radix selection on the
//     FP32 bit patterns (11 + 11 + 9 bits). The Sampson error is evaluated
//     without cancellation: with m1 = m0 + d (d = flow / f, third component 0)
//     and R m0 = m0 + Q m0, the epipolar residual is
//         t . (m0 x d + (Q m0) x m1),
//     a sum of small terms, where m1^T E m0 would cancel O(1) products.
//  4. k_epi_argmin: the smallest median (lowest sample on ties).
//  5. Reweighted least squares: inliers of the winner (error <= (2.5 s)^2,
//     s = 1.4826 (1 + 5 / (n - 8)) sqrt(median)), A^T A of their rows
//     m1 (x) m0 in FP64 (per-block partials reduced in a fixed order), its
//     smallest eigenvector by inverse iteration, projected again.
//  6. The four decompositions; k_epi_cheirality counts the valid pixels whose
//     triangulated depth is positive in both cameras; the first candidate with
//     the largest count gives T_1, with |t| = the caller's baseline.
#include <cmath>

#include "voldor_internal.cuh"

namespace vd {

constexpr int kEpiSampleBlock = 64;
constexpr int kEpiSamplesPerBlock = 8;      // samples per histogram block
constexpr int kEpiBins = 2048;
constexpr int kEpiThreads = 256;

// ---------------------------------------------------------------------------
// 1. Records (and the count of valid pixels into info[2])
// ---------------------------------------------------------------------------
__device__ __forceinline__ bool epi_target_inside(const DevParams& p, const DevState& s, int j)
{
    const float2 f = load_flow(s.flows, p.flow_f16, (size_t)j);
    const double u = (double)(j % p.W) + (double)f.x, v = (double)(j / p.W) + (double)f.y;
    return u >= 0.0 && u <= (double)(p.W - 1) && v >= 0.0 && v <= (double)(p.H - 1);
}

__global__ void k_epi_records(DevParams p, DevState s, EpiState e)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    const int cnt = __syncthreads_count(j < p.N && epi_target_inside(p, s, j));
    if (threadIdx.x == 0 && cnt) atomicAdd(reinterpret_cast<unsigned long long*>(e.info + 2), (unsigned long long)cnt);
    if (j >= p.N) return;
    const int x = j % p.W, y = j / p.W;
    const float2 f = load_flow(s.flows, p.flow_f16, (size_t)j);
    const double u = (double)x + (double)f.x, v = (double)y + (double)f.y;
    float4 r;
    if (u >= 0.0 && u <= (double)(p.W - 1) && v >= 0.0 && v <= (double)(p.H - 1)) {
        r.x = (float)(((double)x - p.cxd) / p.fxd);
        r.y = (float)(((double)y - p.cyd) / p.fyd);
        r.z = (float)((double)f.x / p.fxd);
        r.w = (float)((double)f.y / p.fyd);
    } else {
        r.x = __int_as_float(0x7fc00000);
        r.y = r.z = r.w = 0.f;
    }
    e.rec[j] = r;
}

// ---------------------------------------------------------------------------
// FP64 helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ void cross3d(const double* a, const double* b, double* o)
{
    o[0] = a[1] * b[2] - a[2] * b[1];
    o[1] = a[2] * b[0] - a[0] * b[2];
    o[2] = a[0] * b[1] - a[1] * b[0];
}

__device__ __forceinline__ bool unit3d(double* a)
{
    const double n = sqrt(a[0] * a[0] + a[1] * a[1] + a[2] * a[2]);
    if (!(n > 0.0)) return false;
    a[0] /= n; a[1] /= n; a[2] /= n;
    return true;
}

// Symmetric 3 x 3 eigen-decomposition by cyclic Jacobi rotations (two-sided):
// A (row-major) is overwritten; columns of V are the eigenvectors, d the values.
__device__ void sym3_eigen(double* A, double* d, double* V)
{
    for (int i = 0; i < 9; ++i) V[i] = (i % 4 == 0) ? 1.0 : 0.0;
    for (int sweep = 0; sweep < 30; ++sweep) {
        const double off = A[1] * A[1] + A[2] * A[2] + A[5] * A[5];
        const double dia = A[0] * A[0] + A[4] * A[4] + A[8] * A[8];
        if (!(off > 1e-32 * dia)) break;
        for (int pq = 0; pq < 3; ++pq) {
            const int pp = pq == 2 ? 1 : 0, qq = pq == 0 ? 1 : 2;
            const double apq = A[pp * 3 + qq];
            if (apq == 0.0) continue;
            const double th = (A[qq * 3 + qq] - A[pp * 3 + pp]) / (2.0 * apq);
            const double t = (th >= 0.0 ? 1.0 : -1.0) / (fabs(th) + sqrt(th * th + 1.0));
            const double c = 1.0 / sqrt(t * t + 1.0), sn = t * c;
            for (int k = 0; k < 3; ++k) {
                const double akp = A[k * 3 + pp], akq = A[k * 3 + qq];
                A[k * 3 + pp] = c * akp - sn * akq;
                A[k * 3 + qq] = sn * akp + c * akq;
            }
            for (int k = 0; k < 3; ++k) {
                const double apk = A[pp * 3 + k], aqk = A[qq * 3 + k];
                A[pp * 3 + k] = c * apk - sn * aqk;
                A[qq * 3 + k] = sn * apk + c * aqk;
            }
            for (int k = 0; k < 3; ++k) {
                const double vkp = V[k * 3 + pp], vkq = V[k * 3 + qq];
                V[k * 3 + pp] = c * vkp - sn * vkq;
                V[k * 3 + qq] = sn * vkp + c * vkq;
            }
        }
    }
    d[0] = A[0]; d[1] = A[4]; d[2] = A[8];
}

// Projection onto the essential matrices, E = U diag(1, 1, 0) V^T with
// det U = det V = +1, from the eigenvectors of Ein^T Ein. False if rank < 2.
// Kept out of line: inlined into k_epi_samples by nvcc 13.0 it returned false
// for valid input, while the same code called out of line (and a line-by-line
// NumPy replay) returns the correct projection; the cause was not found.
__device__ __noinline__ bool essential_project(const double* Ein, double* E, double* U, double* V)
{
    double A[9], d[3], Q[9];
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b)
            A[a * 3 + b] = Ein[a] * Ein[b] + Ein[3 + a] * Ein[3 + b] + Ein[6 + a] * Ein[6 + b];
    sym3_eigen(A, d, Q);
    int o0 = 0, o1 = 1, o2 = 2;                       // descending order of d
    if (d[o0] < d[o1]) { const int t = o0; o0 = o1; o1 = t; }
    if (d[o1] < d[o2]) { const int t = o1; o1 = o2; o2 = t; }
    if (d[o0] < d[o1]) { const int t = o0; o0 = o1; o1 = t; }
    double v[3][3], u[3][3];
    const int oi[2] = {o0, o1};
    for (int i = 0; i < 2; ++i)
        for (int k = 0; k < 3; ++k) v[i][k] = Q[k * 3 + oi[i]];
    cross3d(v[0], v[1], v[2]);
    for (int i = 0; i < 2; ++i) {
        for (int r = 0; r < 3; ++r) u[i][r] = Ein[r * 3 + 0] * v[i][0] + Ein[r * 3 + 1] * v[i][1] + Ein[r * 3 + 2] * v[i][2];
        if (!unit3d(u[i])) return false;
    }
    // u_1 is orthogonal to u_0 in exact arithmetic; re-orthogonalise
    const double dd = u[0][0] * u[1][0] + u[0][1] * u[1][1] + u[0][2] * u[1][2];
    for (int r = 0; r < 3; ++r) u[1][r] -= dd * u[0][r];
    if (!unit3d(u[1])) return false;
    cross3d(u[0], u[1], u[2]);
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) {
            U[r * 3 + c] = u[c][r];
            V[r * 3 + c] = v[c][r];
            E[r * 3 + c] = u[0][r] * v[0][c] + u[1][r] * v[1][c];
        }
    return true;
}

// R = U W V^T (a = 0) or U W^T V^T (a = 1), W = [[0,-1,0],[1,0,0],[0,0,1]].
__device__ void rot_candidate(const double* U, const double* V, int a, double* R)
{
    // U W: columns (u1, -u0, u2); U W^T: columns (-u1, u0, u2)
    double UW[9];
    for (int r = 0; r < 3; ++r) {
        UW[r * 3 + 0] = a == 0 ? U[r * 3 + 1] : -U[r * 3 + 1];
        UW[r * 3 + 1] = a == 0 ? -U[r * 3 + 0] : U[r * 3 + 0];
        UW[r * 3 + 2] = U[r * 3 + 2];
    }
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c)
            R[r * 3 + c] = UW[r * 3 + 0] * V[c * 3 + 0] + UW[r * 3 + 1] * V[c * 3 + 1] + UW[r * 3 + 2] * V[c * 3 + 2];
}

// Scoring form of an essential matrix: the rotation candidate with the larger
// trace (the smaller angle) as Q = R - I, and t = u_2.
__device__ void scoring_form(const double* U, const double* V, float* f)
{
    double Ra[9], Rb[9];
    rot_candidate(U, V, 0, Ra);
    rot_candidate(U, V, 1, Rb);
    const double* R = (Ra[0] + Ra[4] + Ra[8] >= Rb[0] + Rb[4] + Rb[8]) ? Ra : Rb;
    for (int i = 0; i < 9; ++i) f[i] = (float)(R[i] - ((i % 4 == 0) ? 1.0 : 0.0));
    for (int r = 0; r < 3; ++r) f[9 + r] = (float)U[r * 3 + 2];
}

// ---------------------------------------------------------------------------
// 2. Minimal samples
// ---------------------------------------------------------------------------
__global__ void k_epi_samples(DevParams p, DevState s, EpiState e)
{
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= e.M) return;
    int ok = 1, why = 1;
    long long j[8];
    for (int q = 0; q < 2; ++q) {
        const U64x4 r = philox4x64_10((uint64_t)m, (uint64_t)q, 0, (uint64_t)kStreamEpi, p.seed, p.window_id);
        for (int i = 0; i < 4; ++i) j[4 * q + i] = (long long)__umul64hi(r.v[i], (uint64_t)p.N);
    }
    for (int a = 0; a < 8; ++a)
        for (int b = a + 1; b < 8; ++b)
            if (j[a] == j[b]) { ok = 0; why = -1; }
    double A[8][9];
    for (int i = 0; i < 8 && ok; ++i) {
        const int x = (int)(j[i] % p.W), y = (int)(j[i] / p.W);
        const float2 f = load_flow(s.flows, p.flow_f16, (size_t)j[i]);
        const double u = (double)x + (double)f.x, v = (double)y + (double)f.y;
        if (!(u >= 0.0 && u <= (double)(p.W - 1) && v >= 0.0 && v <= (double)(p.H - 1))) { ok = 0; why = -2; break; }
        const double m0[3] = {((double)x - p.cxd) / p.fxd, ((double)y - p.cyd) / p.fyd, 1.0};
        const double m1[3] = {(u - p.cxd) / p.fxd, (v - p.cyd) / p.fyd, 1.0};
        for (int r = 0; r < 3; ++r)
            for (int c = 0; c < 3; ++c) A[i][r * 3 + c] = m1[r] * m0[c];
    }
    double Ev[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    if (ok) {
        // Gaussian elimination with complete pivoting; col[] tracks the column order
        int col[9];
        for (int c = 0; c < 9; ++c) col[c] = c;
        double piv0 = 0.0;
        for (int k = 0; k < 8 && ok; ++k) {
            int br = k, bc = k;
            double best = -1.0;
            for (int r = k; r < 8; ++r)
                for (int c = k; c < 9; ++c)
                    if (fabs(A[r][c]) > best) { best = fabs(A[r][c]); br = r; bc = c; }
            if (k == 0) piv0 = best;
            if (!(best > 1e-12 * piv0) || !(best > 0.0)) { ok = 0; why = -3; break; }
            if (br != k)
                for (int c = 0; c < 9; ++c) { const double t = A[k][c]; A[k][c] = A[br][c]; A[br][c] = t; }
            if (bc != k) {
                for (int r = 0; r < 8; ++r) { const double t = A[r][k]; A[r][k] = A[r][bc]; A[r][bc] = t; }
                const int t = col[k]; col[k] = col[bc]; col[bc] = t;
            }
            const double inv = 1.0 / A[k][k];
            for (int r = k + 1; r < 8; ++r) {
                const double f = A[r][k] * inv;
                if (f == 0.0) continue;
                for (int c = k; c < 9; ++c) A[r][c] -= f * A[k][c];
            }
        }
        if (ok) {
            double z[9];
            z[8] = 1.0;
            for (int k = 7; k >= 0; --k) {
                double acc = 0.0;
                for (int c = k + 1; c < 9; ++c) acc += A[k][c] * z[c];
                z[k] = -acc / A[k][k];
            }
            double nn = 0.0;
            for (int c = 0; c < 9; ++c) nn += z[c] * z[c];
            nn = 1.0 / sqrt(nn);
            for (int c = 0; c < 9; ++c) Ev[col[c]] = z[c] * nn;
        }
    }
    double E[9], U[9], V[9];
    if (ok && !essential_project(Ev, E, U, V)) { ok = 0; why = -4; }
    e.valid[m] = why;
    float* f = e.form + (size_t)m * 12;
    if (ok) {
        for (int i = 0; i < 9; ++i) {
            e.E[(size_t)m * 9 + i] = E[i];
            e.UV[(size_t)m * 18 + i] = U[i];
            e.UV[(size_t)m * 18 + 9 + i] = V[i];
        }
        scoring_form(U, V, f);
    } else {
        for (int i = 0; i < 9; ++i) e.E[(size_t)m * 9 + i] = 0.0;
        for (int i = 0; i < 12; ++i) f[i] = 0.f;
    }
}

// ---------------------------------------------------------------------------
// 3. Sampson error (FP32, cancellation-free) and radix selection of the median
// ---------------------------------------------------------------------------
__device__ __forceinline__ float sampson32(const float* F, float4 r)
{
    const float m0x = r.x, m0y = r.y, dx = r.z, dy = r.w;
    const float m1x = m0x + dx, m1y = m0y + dy;
    const float q0 = fmaf(F[0], m0x, fmaf(F[1], m0y, F[2]));
    const float q1 = fmaf(F[3], m0x, fmaf(F[4], m0y, F[5]));
    const float q2 = fmaf(F[6], m0x, fmaf(F[7], m0y, F[8]));
    const float tx = F[9], ty = F[10], tz = F[11];
    // c = m0 x d + q x m1
    const float cx = -dy + (q1 - q2 * m1y);
    const float cy = dx + (q2 * m1x - q0);
    const float cz = fmaf(m0x, dy, -m0y * dx) + fmaf(q0, m1y, -q1 * m1x);
    const float e = fmaf(tx, cx, fmaf(ty, cy, tz * cz));
    // E m0 = t x (m0 + q)
    const float rx = m0x + q0, ry = m0y + q1, rz = 1.f + q2;
    const float a0 = fmaf(ty, rz, -tz * ry), a1 = fmaf(tz, rx, -tx * rz);
    // E^T m1 = -R^T (t x m1), R = I + Q
    const float w0 = fmaf(ty, 1.f, -tz * m1y), w1 = fmaf(tz, m1x, -tx), w2 = fmaf(tx, m1y, -ty * m1x);
    const float b0 = w0 + fmaf(F[0], w0, fmaf(F[3], w1, F[6] * w2));
    const float b1 = w1 + fmaf(F[1], w0, fmaf(F[4], w1, F[7] * w2));
    const float den = fmaf(a0, a0, fmaf(a1, a1, fmaf(b0, b0, b1 * b1)));
    const float d = e * e / den;
    return (den > 0.f && d == d) ? d : __int_as_float(0x7f800000);
}

__device__ __forceinline__ int epi_digit(unsigned bits, int pass)
{
    return pass == 0 ? (int)(bits >> 20) : pass == 1 ? (int)((bits >> 9) & 0x7ff) : (int)(bits & 0x1ff);
}

__device__ __forceinline__ bool epi_prefix_match(unsigned bits, int pass, unsigned prefix)
{
    return pass == 0 || (pass == 1 ? (bits >> 20) == prefix : (bits >> 9) == prefix);
}

// grid (pixel chunks, M / 8); dynamic shared memory 8 x kEpiBins counters.
__global__ void __launch_bounds__(kEpiThreads, 2) k_epi_hist(DevParams p, EpiState e, int pass)
{
    extern __shared__ unsigned h[];
    __shared__ float F[kEpiSamplesPerBlock][12];
    __shared__ unsigned pre[kEpiSamplesPerBlock];
    __shared__ int act[kEpiSamplesPerBlock];
    const int m0 = blockIdx.y * kEpiSamplesPerBlock;
    for (int i = threadIdx.x; i < kEpiSamplesPerBlock * kEpiBins; i += blockDim.x) h[i] = 0;
    if (threadIdx.x < kEpiSamplesPerBlock * 12) {
        const int sm = threadIdx.x / 12, q = threadIdx.x % 12;
        F[sm][q] = (m0 + sm < e.M) ? e.form[(size_t)(m0 + sm) * 12 + q] : 0.f;
    }
    if (threadIdx.x < kEpiSamplesPerBlock) {
        const int m = m0 + threadIdx.x;
        act[threadIdx.x] = (m < e.M && e.valid[m] > 0) ? 1 : 0;
        pre[threadIdx.x] = (m < e.M) ? e.prefix[m] : 0u;
    }
    __syncthreads();
    const long long lo = (long long)p.N * blockIdx.x / gridDim.x;
    const long long hi = (long long)p.N * (blockIdx.x + 1) / gridDim.x;
    auto count = [&](const float4& r) {
        if (r.x != r.x) return;                       // invalid pixel
#pragma unroll
        for (int sm = 0; sm < kEpiSamplesPerBlock; ++sm) {
            if (!act[sm]) continue;
            const unsigned bits = __float_as_uint(sampson32(F[sm], r));
            if (!epi_prefix_match(bits, pass, pre[sm])) continue;
            atomicAdd(&h[sm * kEpiBins + epi_digit(bits, pass)], 1u);
        }
    };
    // two records in flight per thread
    long long j = lo + threadIdx.x;
    for (; j + blockDim.x < hi; j += 2 * blockDim.x) {
        const float4 r0 = e.rec[j], r1 = e.rec[j + blockDim.x];
        count(r0);
        count(r1);
    }
    if (j < hi) count(e.rec[j]);
    __syncthreads();
    unsigned* g = e.hist + (size_t)pass * e.M * kEpiBins;
    for (int i = threadIdx.x; i < kEpiSamplesPerBlock * kEpiBins; i += blockDim.x) {
        const int sm = i / kEpiBins, b = i % kEpiBins;
        if (m0 + sm < e.M && h[i]) atomicAdd(g + (size_t)(m0 + sm) * kEpiBins + b, h[i]);
    }
}

// One warp per sample: the bin of this pass that holds the remaining rank.
__global__ void k_epi_select(EpiState e, int pass)
{
    const int lane = threadIdx.x & 31;
    const int m = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (m >= e.M) return;
    if (e.valid[m] <= 0 || e.info[2] == 0) {
        if (lane == 0) e.median[m] = __int_as_float(0x7f800000);
        return;
    }
    const unsigned rank = pass == 0 ? (unsigned)((e.info[2] - 1) / 2) : e.rank[m];
    const unsigned* h = e.hist + ((size_t)pass * e.M + m) * kEpiBins;
    const int nb = pass == 2 ? 512 : kEpiBins;
    const int per = nb / 32;
    unsigned mine = 0;
    for (int i = 0; i < per; ++i) mine += h[lane * per + i];
    unsigned incl = mine;
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += v;
    }
    const unsigned excl = incl - mine;
    const bool here = rank >= excl && rank < incl;
    const unsigned ball = __ballot_sync(0xffffffffu, here);
    if (!ball) {                                      // counts do not reach the rank: no valid value
        if (lane == 0) e.median[m] = __int_as_float(0x7f800000);
        return;
    }
    const int L = __ffs(ball) - 1;
    if (lane == L) {
        unsigned cum = excl;
        int b = lane * per;
        for (; b < lane * per + per - 1 && cum + h[b] <= rank; ++b) cum += h[b];
        const unsigned prefix = e.prefix[m];
        if (pass == 0) { e.prefix[m] = (unsigned)b; e.rank[m] = rank - cum; }
        else if (pass == 1) { e.prefix[m] = (prefix << 11) | (unsigned)b; e.rank[m] = rank - cum; }
        else e.median[m] = __uint_as_float((prefix << 9) | (unsigned)b);
    }
}

// ---------------------------------------------------------------------------
// 4. Winner
// ---------------------------------------------------------------------------
__global__ void k_epi_argmin(EpiState e)
{
    float best = __int_as_float(0x7f800000);
    int bi = 0x7fffffff;
    for (int m = threadIdx.x; m < e.M; m += blockDim.x) {
        const float v = e.median[m];
        if (v < best || (v == best && m < bi)) { best = v; bi = m; }
    }
    for (int o = 16; o > 0; o >>= 1) {
        const float ov = __shfl_xor_sync(0xffffffffu, best, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ov < best || (ov == best && oi < bi)) { best = ov; bi = oi; }
    }
    __shared__ float wv[32];
    __shared__ int wi[32];
    if ((threadIdx.x & 31) == 0) { wv[threadIdx.x >> 5] = best; wi[threadIdx.x >> 5] = bi; }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w)
            if (wv[w] < best || (wv[w] == best && wi[w] < bi)) { best = wv[w]; bi = wi[w]; }
        const bool any = best < __int_as_float(0x7f800000);
        e.info[0] = any ? bi : -1;
    }
}

// ---------------------------------------------------------------------------
// 5. Reweighted least squares
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kEpiThreads) k_epi_refine_accum(DevParams p, DevState s, EpiState e)
{
    __shared__ float F[12];
    __shared__ float thr;
    const long long best = e.info[0];
    if (best < 0) return;
    if (threadIdx.x < 12) F[threadIdx.x] = e.form[best * 12 + threadIdx.x];
    if (threadIdx.x == 0) {
        const double n = (double)e.info[2];
        const double sc = 1.4826 * (1.0 + 5.0 / fmax(n - 8.0, 1.0)) * sqrt((double)e.median[best]);
        thr = (float)((2.5 * sc) * (2.5 * sc));
    }
    __syncthreads();
    double acc[46];
    for (int i = 0; i < 46; ++i) acc[i] = 0.0;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < p.N; j += gridDim.x * blockDim.x) {
        const float4 r = e.rec[j];
        if (r.x != r.x || !(sampson32(F, r) <= thr)) continue;
        const int x = j % p.W, y = j / p.W;
        const float2 f = load_flow(s.flows, p.flow_f16, (size_t)j);
        const double m0[3] = {((double)x - p.cxd) / p.fxd, ((double)y - p.cyd) / p.fyd, 1.0};
        const double m1[3] = {((double)x + (double)f.x - p.cxd) / p.fxd, ((double)y + (double)f.y - p.cyd) / p.fyd, 1.0};
        double a[9];
        for (int rr = 0; rr < 3; ++rr)
            for (int c = 0; c < 3; ++c) a[rr * 3 + c] = m1[rr] * m0[c];
        int k = 0;
        for (int u = 0; u < 9; ++u)
            for (int v = u; v < 9; ++v) acc[k++] += a[u] * a[v];
        acc[45] += 1.0;
    }
    // block reduction in a fixed order: warps by shuffles, then warp 0 over warps
    __shared__ double ws[kEpiThreads / 32][46];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int i = 0; i < 46; ++i) {
        double v = acc[i];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) ws[warp][i] = v;
    }
    __syncthreads();
    if (threadIdx.x < 46) {
        double t = 0.0;
        for (int w = 0; w < kEpiThreads / 32; ++w) t += ws[w][threadIdx.x];
        e.partial[(size_t)blockIdx.x * 46 + threadIdx.x] = t;
    }
}

// Threads 0..45 sum the partials in block order; thread 0 then takes the
// eigenvector of the smallest eigenvalue of the 9 x 9 A^T A by inverse
// iteration started at the winning sample's E, through the Cholesky factor of
// A^T A + d I (d = 1e-13 trace: the shift keeps the eigenvectors and makes an
// exactly singular A^T A, as from noiseless flows, factorable), until the
// iterate moves by less than 1e-15 (at most 40 steps; the error shrinks by the
// ratio of the two smallest eigenvalues per step, 0.006 on the driving
// windows). The result is projected again; the four decompositions follow.
__global__ void k_epi_refine_solve(EpiState e)
{
    __shared__ double sum[46];
    const long long best = e.info[0];
    if (best < 0) return;
    if (threadIdx.x < 46) {
        double t = 0.0;
        for (int b = 0; b < e.partial_blocks; ++b) t += e.partial[(size_t)b * 46 + threadIdx.x];
        sum[threadIdx.x] = t;
    }
    __syncthreads();
    if (threadIdx.x != 0) return;
    e.info[3] = (long long)sum[45];
    double E[9], U[9], Vv[9];
    bool ok = false;
    if (sum[45] >= 8.0) {
        double A[81];
        {
            int k = 0;
            for (int u = 0; u < 9; ++u)
                for (int v = u; v < 9; ++v) { A[u * 9 + v] = sum[k]; A[v * 9 + u] = sum[k]; ++k; }
        }
        double tr = 0.0;
        for (int i = 0; i < 9; ++i) tr += A[i * 9 + i];
        const double shift = 1e-13 * tr;
        // Cholesky: A + shift I = L L^T (lower), with the reciprocals of its diagonal
        double L[81], inv[9];
        bool chol = tr > 0.0;
        for (int i = 0; i < 9 && chol; ++i) {
            for (int j = 0; j <= i; ++j) {
                double acc = A[i * 9 + j] + (i == j ? shift : 0.0);
                for (int k = 0; k < j; ++k) acc -= L[i * 9 + k] * L[j * 9 + k];
                if (i == j) {
                    if (!(acc > 0.0)) { chol = false; break; }
                    L[i * 9 + i] = sqrt(acc);
                    inv[i] = 1.0 / L[i * 9 + i];
                } else {
                    L[i * 9 + j] = acc * inv[j];
                }
            }
        }
        if (chol) {
            double x[9];
            for (int i = 0; i < 9; ++i) x[i] = e.E[best * 9 + i];
            for (int it = 0; it < 40; ++it) {
                double y[9], z[9];
#pragma unroll
                for (int i = 0; i < 9; ++i) {                  // L y = x
                    double acc = x[i];
#pragma unroll
                    for (int k = 0; k < i; ++k) acc -= L[i * 9 + k] * y[k];
                    y[i] = acc * inv[i];
                }
#pragma unroll
                for (int i = 8; i >= 0; --i) {                 // L^T z = y
                    double acc = y[i];
#pragma unroll
                    for (int k = i + 1; k < 9; ++k) acc -= L[k * 9 + i] * z[k];
                    z[i] = acc * inv[i];
                }
                double nz = 0.0;
#pragma unroll
                for (int i = 0; i < 9; ++i) nz += z[i] * z[i];
                nz = 1.0 / sqrt(nz);
                double step = 0.0;
#pragma unroll
                for (int i = 0; i < 9; ++i) {
                    const double zi = z[i] * nz;
                    step += (zi - x[i]) * (zi - x[i]);
                    x[i] = zi;
                }
                if (step < 1e-30) break;
            }
            ok = essential_project(x, E, U, Vv);
        }
    }
    if (!ok)
        for (int i = 0; i < 9; ++i) {
            E[i] = e.E[best * 9 + i];
            U[i] = e.UV[best * 18 + i];
            Vv[i] = e.UV[best * 18 + 9 + i];
        }
    for (int i = 0; i < 9; ++i) { e.refined[i] = E[i]; e.refined[9 + i] = U[i]; e.refined[18 + i] = Vv[i]; }
    for (int a = 0; a < 2; ++a) {
        double R[9];
        rot_candidate(U, Vv, a, R);
        for (int sg = 0; sg < 2; ++sg) {
            double* o = e.cand + (2 * a + sg) * 12;
            for (int r = 0; r < 3; ++r) {
                for (int c = 0; c < 3; ++c) o[r * 4 + c] = R[r * 3 + c];
                o[r * 4 + 3] = (sg == 0 ? 1.0 : -1.0) * U[r * 3 + 2];
            }
        }
    }
    for (int i = 0; i < 4; ++i) e.info[4 + i] = 0;
}

// ---------------------------------------------------------------------------
// 6. Cheirality and T_1
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kEpiThreads) k_epi_cheirality(DevParams p, DevState s, EpiState e)
{
    __shared__ double Cd[48];
    if (e.info[0] < 0) return;
    if (threadIdx.x < 48) Cd[threadIdx.x] = e.cand[threadIdx.x];
    __syncthreads();
    unsigned cnt[4] = {0, 0, 0, 0};
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < p.N; j += gridDim.x * blockDim.x) {
        if (e.rec[j].x != e.rec[j].x) continue;
        const int x = j % p.W, y = j / p.W;
        const float2 f = load_flow(s.flows, p.flow_f16, (size_t)j);
        const double m0x = ((double)x - p.cxd) / p.fxd, m0y = ((double)y - p.cyd) / p.fyd;
        const double m1x = ((double)x + (double)f.x - p.cxd) / p.fxd, m1y = ((double)y + (double)f.y - p.cyd) / p.fyd;
        for (int i = 0; i < 4; ++i) {
            const double* T = Cd + 12 * i;
            const double Rx = T[0] * m0x + T[1] * m0y + T[2];
            const double Ry = T[4] * m0x + T[5] * m0y + T[6];
            const double Rz = T[8] * m0x + T[9] * m0y + T[10];
            const double ax = Rx - m1x * Rz, bx = m1x * T[11] - T[3];
            const double ay = Ry - m1y * Rz, by = m1y * T[11] - T[7];
            const double aa = ax * ax + ay * ay, ab = ax * bx + ay * by;
            if (!(aa > 0.0) || !(ab > 0.0)) continue;
            const double z1 = (ab / aa) * Rz + T[11];
            if (z1 > 0.0) ++cnt[i];
        }
    }
    for (int i = 0; i < 4; ++i) {
        unsigned v = cnt[i];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if ((threadIdx.x & 31) == 0 && v) atomicAdd((unsigned long long*)(e.info + 4 + i), (unsigned long long)v);
    }
}

__global__ void k_epi_finish(EpiState e, double baseline)
{
    if (threadIdx.x != 0 || e.info[0] < 0) return;
    int c = 0;
    for (int i = 1; i < 4; ++i)
        if (e.info[4 + i] > e.info[4 + c]) c = i;
    e.info[1] = c;
    const double* T = e.cand + 12 * c;
    for (int r = 0; r < 3; ++r) {
        for (int q = 0; q < 3; ++q) e.T1[r * 4 + q] = T[r * 4 + q];
        e.T1[r * 4 + 3] = baseline * T[r * 4 + 3];
    }
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
static int epi_refine_blocks() { return 2 * 152; }

// Carves the scratch for M samples out of `base` (which may be null to measure)
// and returns the bytes it spans; every piece starts on a 256-byte boundary.
size_t epi_layout(void* base, int M, float4* rec, EpiState* e)
{
    const uintptr_t start = reinterpret_cast<uintptr_t>(base);
    size_t off = 0;
    auto take = [&](size_t n) {
        void* r = reinterpret_cast<void*>(start + off);
        off += (n + 255) & ~(size_t)255;
        return r;
    };
    e->M = M;
    e->rec = rec;
    e->valid = static_cast<int*>(take((size_t)M * 4));
    e->E = static_cast<double*>(take((size_t)M * 9 * 8));
    e->UV = static_cast<double*>(take((size_t)M * 18 * 8));
    e->form = static_cast<float*>(take((size_t)M * 12 * 4));
    e->hist = static_cast<unsigned*>(take((size_t)3 * M * kEpiBins * 4));
    e->prefix = static_cast<unsigned*>(take((size_t)M * 4));
    e->rank = static_cast<unsigned*>(take((size_t)M * 4));
    e->median = static_cast<float*>(take((size_t)M * 4));
    e->info = static_cast<long long*>(take(8 * 8));
    e->partial_blocks = epi_refine_blocks();
    e->partial = static_cast<double*>(take((size_t)e->partial_blocks * 46 * 8));
    e->refined = static_cast<double*>(take(27 * 8));
    e->cand = static_cast<double*>(take(48 * 8));
    e->T1 = static_cast<double*>(take(12 * 8));
    return off;
}

size_t epi_scratch_bytes(int M)
{
    EpiState e;
    return epi_layout(nullptr, M, nullptr, &e);
}

// Enqueues the whole estimate on st; returns the number of kernels launched.
int launch_epipolar(const DevParams& p, const DevState& s, const EpiState& e, double baseline, cudaStream_t st)
{
    static bool attr = false;
    const int hist_smem = kEpiSamplesPerBlock * kEpiBins * 4;
    if (!attr) {
        cudaFuncSetAttribute(k_epi_hist, cudaFuncAttributeMaxDynamicSharedMemorySize, hist_smem);
        attr = true;
    }
    int k = 0;
    cudaMemsetAsync(e.hist, 0, (size_t)3 * e.M * kEpiBins * 4, st);
    cudaMemsetAsync(e.prefix, 0, (size_t)e.M * 4, st);
    cudaMemsetAsync(e.info, 0, 8 * 8, st);
    k_epi_records<<<(p.N + 255) / 256, 256, 0, st>>>(p, s, e); ++k;
    k_epi_samples<<<(e.M + kEpiSampleBlock - 1) / kEpiSampleBlock, kEpiSampleBlock, 0, st>>>(p, s, e); ++k;
    const int groups = (e.M + kEpiSamplesPerBlock - 1) / kEpiSamplesPerBlock;
    int chunks = (8 * 152 + groups - 1) / groups;
    chunks = chunks < 1 ? 1 : (chunks > 1024 ? 1024 : chunks);
    for (int pass = 0; pass < 3; ++pass) {
        k_epi_hist<<<dim3(chunks, groups), kEpiThreads, hist_smem, st>>>(p, e, pass); ++k;
        k_epi_select<<<(e.M + 7) / 8, 256, 0, st>>>(e, pass); ++k;
    }
    k_epi_argmin<<<1, 1024, 0, st>>>(e); ++k;
    k_epi_refine_accum<<<e.partial_blocks, kEpiThreads, 0, st>>>(p, s, e); ++k;
    k_epi_refine_solve<<<1, 64, 0, st>>>(e); ++k;
    k_epi_cheirality<<<epi_refine_blocks(), kEpiThreads, 0, st>>>(p, s, e); ++k;
    k_epi_finish<<<1, 32, 0, st>>>(e, baseline); ++k;
    return k;
}

}  // namespace vd
