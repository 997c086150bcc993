// Absolute scale from the ground plane (Sec. 6.1: the mode over the pixels
// whose surface normal is near the vertical).
//
//  k_ground_hist: per interior pixel of I_0 (FP64), the back-projected point
//    P = theta K^-1 [x y 1]^T and the unit normal of the cross product of the
//    central differences of its horizontal and vertical neighbours (its sign
//    does not matter: only |n_y| and |n . P| are used); a rigid pixel (mean W >= 1/2) below the camera (P_y > 0)
//    whose normal is within max_tilt of the camera's y axis, with all five depths
//    strictly inside the depth range, adds |n . P| (its tangent plane's distance
//    from the camera) to a 4096-bin histogram of log2 height over [-8, 8)
//    (shared-memory counts per block, then global atomics).
//  k_ground_mode: one block: the argmax of the 5-bin box-filtered histogram
//    (lowest bin on ties), the count-weighted mean of the bin centres of the raw
//    histogram over the 5 bins around it, and scale = camera height / 2^mode.
//  k_ground_apply: optionally multiplies the depth and every translation by
//    the scale.
#include <cmath>

#include "voldor_internal.cuh"

namespace vd {

constexpr int kGroundBins = 4096;
constexpr double kGroundLo = -8.0, kGroundHi = 8.0;

__global__ void __launch_bounds__(256) k_ground_hist(DevParams p, DevState s, double cos_tilt, double dmin,
                                                     double dmax, unsigned* hist)
{
    __shared__ unsigned h[kGroundBins];
    for (int i = threadIdx.x; i < kGroundBins; i += blockDim.x) h[i] = 0;
    __syncthreads();
    const double binw = (kGroundHi - kGroundLo) / kGroundBins;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < p.N; j += gridDim.x * blockDim.x) {
        const int x = j % p.W, y = j / p.W;
        if (x < 1 || y < 1 || x > p.W - 2 || y > p.H - 2) continue;
        const double th = s.theta[j], tl = s.theta[j - 1], tr = s.theta[j + 1];
        const double tu = s.theta[j - p.W], td = s.theta[j + p.W];
        if (!(th > dmin && th < dmax && tl > dmin && tl < dmax && tr > dmin && tr < dmax && tu > dmin &&
              tu < dmax && td > dmin && td < dmax))
            continue;
        float wsum = 0.f;
        for (int t = 0; t < p.T; ++t) wsum += s.wmap[(size_t)t * p.N + j];
        if (!(wsum >= 0.5f * (float)p.T)) continue;
        const double dx = ((double)x - p.cxd) / p.fxd, dy = ((double)y - p.cyd) / p.fyd;
        const double Px = th * dx, Py = th * dy, Pz = th;
        if (!(Py > 0.0)) continue;
        const double dxl = ((double)(x - 1) - p.cxd) / p.fxd, dxr = ((double)(x + 1) - p.cxd) / p.fxd;
        const double dyu = ((double)(y - 1) - p.cyd) / p.fyd, dyd = ((double)(y + 1) - p.cyd) / p.fyd;
        // a = P(x+1, y) - P(x-1, y), c = P(x, y+1) - P(x, y-1)
        const double ax = tr * dxr - tl * dxl, ay = (tr - tl) * dy, az = tr - tl;
        const double cx = (td - tu) * dx, cy = td * dyd - tu * dyu, cz = td - tu;
        double nx = ay * cz - az * cy, ny = az * cx - ax * cz, nz = ax * cy - ay * cx;
        const double nn = sqrt(nx * nx + ny * ny + nz * nz);
        if (!(nn > 0.0)) continue;
        nx /= nn; ny /= nn; nz /= nn;
        const double np = nx * Px + ny * Py + nz * Pz;
        if (!(fabs(ny) >= cos_tilt)) continue;
        const double hgt = fabs(np);
        if (!(hgt > 0.0)) continue;
        const double l = log2(hgt);
        if (!(l >= kGroundLo && l < kGroundHi)) continue;
        int bin = (int)floor((l - kGroundLo) / binw);
        bin = bin < 0 ? 0 : (bin >= kGroundBins ? kGroundBins - 1 : bin);
        atomicAdd(&h[bin], 1u);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < kGroundBins; i += blockDim.x)
        if (h[i]) atomicAdd(hist + i, h[i]);
}

// out[0] = scale (0 if no candidate), out[1] = mode (log2 height), out[2] = candidates
__global__ void k_ground_mode(const unsigned* hist, double camera_height, double* out)
{
    __shared__ unsigned long long best[1024];
    __shared__ int besti[1024];
    __shared__ unsigned long long total_s[1024];
    unsigned long long bv = 0, tot = 0;
    int bi = 0x7fffffff;
    for (int i = threadIdx.x; i < kGroundBins; i += blockDim.x) {
        unsigned long long sm = 0;
        for (int k = -2; k <= 2; ++k)
            if (i + k >= 0 && i + k < kGroundBins) sm += hist[i + k];
        tot += hist[i];
        if (sm > bv || (sm == bv && i < bi)) { bv = sm; bi = i; }
    }
    best[threadIdx.x] = bv;
    besti[threadIdx.x] = bi;
    total_s[threadIdx.x] = tot;
    __syncthreads();
    if (threadIdx.x != 0) return;
    unsigned long long n = 0;
    for (int t = 0; t < (int)blockDim.x; ++t) {
        n += total_s[t];
        if (best[t] > bv || (best[t] == bv && besti[t] < bi)) { bv = best[t]; bi = besti[t]; }
    }
    out[2] = (double)n;
    if (n == 0) { out[0] = 0.0; out[1] = 0.0; return; }
    const double binw = (kGroundHi - kGroundLo) / kGroundBins;
    double num = 0.0, cnt = 0.0;
    for (int k = -2; k <= 2; ++k)
        if (bi + k >= 0 && bi + k < kGroundBins) {
            num += (double)hist[bi + k] * (kGroundLo + (bi + k + 0.5) * binw);
            cnt += (double)hist[bi + k];
        }
    const double mode = num / cnt;
    out[1] = mode;
    out[0] = camera_height / exp2(mode);
}

__global__ void k_ground_apply(DevParams p, DevState s, const double* out)
{
    const double sc = out[0];
    if (!(sc > 0.0)) return;
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j < p.N) s.theta[j] = (float)((double)s.theta[j] * sc);
    if (j < p.T) {
        s.poses[j * 12 + 3] *= sc;
        s.poses[j * 12 + 7] *= sc;
        s.poses[j * 12 + 11] *= sc;
    }
}

// Enqueues the estimate (and the rescaling if apply); out[3] doubles on the device.
int launch_ground_scale(const DevParams& p, const DevState& s, double camera_height, double cos_tilt, double dmin,
                        double dmax, int apply, unsigned* hist, double* out, cudaStream_t st)
{
    cudaMemsetAsync(hist, 0, kGroundBins * sizeof(unsigned), st);
    const int nb = (p.N + 255) / 256 < 2 * 152 ? (p.N + 255) / 256 : 2 * 152;
    k_ground_hist<<<nb, 256, 0, st>>>(p, s, cos_tilt, dmin, dmax, hist);
    k_ground_mode<<<1, 1024, 0, st>>>(hist, camera_height, out);
    int k = 2;
    if (apply) {
        k_ground_apply<<<(p.N + 255) / 256, 256, 0, st>>>(p, s, out);
        ++k;
    }
    return k;
}

}  // namespace vd
