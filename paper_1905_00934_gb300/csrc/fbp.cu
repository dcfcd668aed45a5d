// Filtered backprojection (FBP) and the CDM-FBP comparison method (Sec. 2, Sec. 4): per-ray
// decomposition into Compton and PE line integrals followed by FBP of each basis.
//
// FBP is the textbook algorithm with the band-limited ramp filter on the projector's geometry
// (parallel beam over pi or 2 pi; flat-detector fan beam over 2 pi):
//   filter      Q(n) = gain * (p(n) / 4 - sum_{odd m} p(n - m) / (pi^2 m^2)), one CTA per view row,
//               the row in shared memory, a direct convolution (Nb/2 taps per output; a few
//               microseconds per slice, so no FFT). Parallel: gain = 1/du. Fan: p pre-weighted by
//               SOD / sqrt(SOD^2 + s^2) on the detector rescaled to the isocentre (s = u SOD/SDD),
//               gain = 1 / (2 du SOD/SDD) (half the ramp).
//   backproject pixel-driven, one thread per pixel, views in shared-memory chunks; the filtered row
//               is read at the pixel's fractional bin (linear interpolation, zero beyond the first
//               and last bin). Parallel: x = (pi/V) sum_v Q_v(k), k = X c/du + Y s/du + k0. Fan:
//               x = (2 pi/V) sum_v Q_v(k) SOD^2 / den^2 with den = SOD - X c - Y s and
//               k = (SDD/du) (Y c - X s) / den + k0.
// The per-view constants are formed in double on the host and rounded once to float.
#include <cuda_runtime.h>
#include <math.h>

#include "dect_internal.cuh"

namespace dect {

constexpr int kFbpFilterThreads = 256;
constexpr int kFbpTileX = 32, kFbpTileY = 8;
constexpr int kFbpViewChunk = 256;

// q[c][v][n]: the filtered rows of sino[c][v][k] (clamp: the CDM constraint p = max(p, 0) on load)
__global__ void __launch_bounds__(kFbpFilterThreads) k_fbp_filter(FbpDev f, const float* __restrict__ sino,
                                                                 float* __restrict__ q, int clamp) {
    extern __shared__ float sh[];
    const int nb = f.nb, half = (nb + 1) / 2;
    float* row = sh;         // [nb]
    float* cw = sh + nb;     // [half]: 1 / (pi^2 (2j+1)^2)
    const size_t base = ((size_t)blockIdx.y * f.nv + blockIdx.x) * nb;
    for (int k = threadIdx.x; k < nb; k += blockDim.x) {
        float p = __ldg(sino + base + k);
        if (clamp) p = fmaxf(p, 0.0f);
        if (f.prew) p *= __ldg(f.prew + k);
        row[k] = p;
    }
    for (int j = threadIdx.x; j < half; j += blockDim.x) {
        const double m = 2.0 * j + 1.0;
        cw[j] = (float)(1.0 / (M_PI * M_PI * m * m));
    }
    __syncthreads();
    for (int n = threadIdx.x; n < nb; n += blockDim.x) {
        // taps at n - m (left) and n + m (right) for odd m = 2j + 1, in increasing m
        float left = 0.0f, right = 0.0f;
        const int jl = (n + 1) / 2, jr = (nb - n) / 2;  // odd m <= n, odd m <= nb - 1 - n
        const int jm = max(jl, jr);
        for (int j = 0; j < jm; ++j) {
            const int m = 2 * j + 1;
            const float w = cw[j];
            if (j < jl) left = fmaf(w, row[n - m], left);
            if (j < jr) right = fmaf(w, row[n + m], right);
        }
        q[base + n] = f.gain * (0.25f * row[n] - (left + right));
    }
}

__global__ void __launch_bounds__(kFbpTileX * kFbpTileY) k_fbp_backproject(FbpDev f, const float* __restrict__ q,
                                                                          float* __restrict__ x, int nch) {
    __shared__ float4 vt[kFbpViewChunk];
    const int i = blockIdx.x * kFbpTileX + threadIdx.x, j = blockIdx.y * kFbpTileY + threadIdx.y;
    const int tid = threadIdx.y * kFbpTileX + threadIdx.x;
    const float X = ((float)i - f.cx) * f.pix, Y = ((float)j - f.cy) * f.pix;
    const int nb = f.nb;
    const size_t chs = (size_t)f.nv * nb;
    const bool inside = i < f.nx && j < f.ny;
    float s0 = 0.0f, s1 = 0.0f;
    for (int v0 = 0; v0 < f.nv; v0 += kFbpViewChunk) {
        const int nvc = min(kFbpViewChunk, f.nv - v0);
        __syncthreads();
        for (int t = tid; t < nvc; t += kFbpTileX * kFbpTileY) vt[t] = __ldg(f.tab + v0 + t);
        __syncthreads();
        for (int t = 0; t < nvc && inside; ++t) {
            const float4 c = vt[t];
            float kf, wgt = 1.0f;
            if (f.fan) {
                const float den = fmaf(-X, c.x, fmaf(-Y, c.y, f.sod));  // SOD - P.n
                const float num = fmaf(Y, c.x, -X * c.y);               // P.e
                const float r = 1.0f / den;
                kf = fmaf(num * r, f.k1, f.k0);
                const float u = f.sod * r;
                wgt = u * u;
            } else {
                kf = fmaf(X, c.x, fmaf(Y, c.y, c.z));
            }
            const float kfl = floorf(kf);
            const int k = (int)kfl;
            if (k < -1 || k > nb - 1) continue;
            const float fr = kf - kfl;
            const float* qv = q + (size_t)(v0 + t) * nb;
            const float a0 = k >= 0 ? __ldg(qv + k) : 0.0f, a1 = k + 1 <= nb - 1 ? __ldg(qv + k + 1) : 0.0f;
            s0 = fmaf(wgt, fmaf(fr, a1 - a0, a0), s0);
            if (nch == 2) {
                const float b0 = k >= 0 ? __ldg(qv + chs + k) : 0.0f, b1 = k + 1 <= nb - 1 ? __ldg(qv + chs + k + 1) : 0.0f;
                s1 = fmaf(wgt, fmaf(fr, b1 - b0, b0), s1);
            }
        }
    }
    if (inside) {
        const size_t e = (size_t)j * f.nx + i;
        x[e] = f.scale * s0;
        if (nch == 2) x[(size_t)f.nx * f.ny + e] = f.scale * s1;
    }
}

// CDM start: a_c = m_l / sum_E S_l f_KN, a_p = 0, mu = mu0 (the decomposition's warm start)
__global__ void k_cdm_start(int64_t n, const float* __restrict__ m_l, float inv_abar, float mu0,
                            float* __restrict__ a_c, float* __restrict__ a_p, float* __restrict__ mu,
                            float* __restrict__ zero) {
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    const float ml = __ldg(m_l + r);
    a_c[r] = ml * inv_abar;
    a_p[r] = 0.0f;
    mu[r] = mu0;
    zero[r] = 0.0f;
}

// planar copies of a slice's measurements {m_h, m_l, w_h, w_l} (the solver keeps them interleaved)
__global__ void k_unpack_meas(int64_t n, const float4* __restrict__ meas, float* __restrict__ planar) {
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    const float4 m = __ldg(meas + r);
    planar[r] = m.x;
    planar[n + r] = m.y;
    planar[2 * n + r] = m.z;
    planar[3 * n + r] = m.w;
}

void launch_unpack_meas(int64_t n, const float4* meas, float* planar, cudaStream_t st) {
    k_unpack_meas<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, meas, planar);
}

void launch_fbp(const FbpDev& f, int nch, const float* sino, float* q, float* x, bool clamp, cudaStream_t st) {
    const size_t smem = sizeof(float) * (f.nb + (f.nb + 1) / 2);
    k_fbp_filter<<<dim3((unsigned)f.nv, (unsigned)nch), kFbpFilterThreads, smem, st>>>(f, sino, q, clamp ? 1 : 0);
    const dim3 grid((unsigned)((f.nx + kFbpTileX - 1) / kFbpTileX), (unsigned)((f.ny + kFbpTileY - 1) / kFbpTileY));
    k_fbp_backproject<<<grid, dim3(kFbpTileX, kFbpTileY), 0, st>>>(f, q, x, nch);
}

void launch_cdm_start(int64_t n, const float* m_l, float inv_abar, float mu0, float* a_c, float* a_p, float* mu,
                      float* zero, cudaStream_t st) {
    k_cdm_start<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, m_l, inv_abar, mu0, a_c, a_p, mu, zero);
}

cudaError_t fbp_init_attributes() {
    // row + odd taps of the largest detector (16384 bins): 96 KB
    return cudaFuncSetAttribute(k_fbp_filter, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)(sizeof(float) * (16384 + 8192)));
}

}  // namespace dect
