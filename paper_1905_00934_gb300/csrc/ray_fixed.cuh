// Fixed-point ray helpers shared by the float32 and float64 projector kernels (the projection
// matrix R of Eq. 2-3 and its transpose): a ray entry is int4 {q0 low word, q0 high word, slope,
// +-w}; a sample's position along the other axis is q0 + t * slope in units of 2^-30 pixel, so R
// and R^T evaluate bit-identical interpolation weights from the same integers.
#pragma once

#include <cuda_runtime.h>

#include "dect_internal.cuh"

namespace dect {

// Fixed-point helpers: a ray entry is {q0 low word, q0 high word, slope, +-w}, q0 and slope in units
// of 2^-30 pixel, with the sign of w giving the axis (negative: sampled per row).
__device__ __forceinline__ long long ray_q0(const int4 P) {
    return ((long long)P.y << 32) | (long long)(unsigned)P.x;
}
__device__ __forceinline__ long long ray_step(const int4 P) { return (long long)P.z; }
__device__ __forceinline__ bool ray_axis(const int4 P) { return P.w < 0; }
__device__ __forceinline__ float ray_w(const int4 P) { return fabsf(__int_as_float(P.w)); }
// position of the sample at index t
__device__ __forceinline__ long long ray_pos(const int4 P, int t) { return ray_q0(P) + (long long)t * P.z; }
// lower interpolation neighbour (floor of the position)
__device__ __forceinline__ int pos_floor(long long q) { return (int)(q >> 30); }
// interpolation weight of the upper neighbour: the top 23 of the 30 fraction bits as a float in [0, 1)
__device__ __forceinline__ float frac_of(long long q) {
    return __uint_as_float(0x3f800000u | (((unsigned)q >> 7) & 0x7fffffu)) - 1.0f;
}

// Index range [lo, hi] along the sampled axis whose positions lie in [-1.5, n_across + 0.5): it
// contains every sample with a non-zero weight (positions in (-1, n_across)) and keeps the lower
// neighbour in [-2, n_across]. Float estimate; the 0.5-pixel margins absorb its rounding.
__device__ __forceinline__ void sample_range(const int4 P, int n_along, int n_across, int& lo, int& hi) {
    const float q0 = (float)P.y * 4294967296.0f + (float)(unsigned)P.x;
    const float q0f = q0 * 9.313225746154785e-10f;  // 2^-30
    const float c1 = (float)P.z * 9.313225746154785e-10f;  // 2^-30
    float a, b;
    if (fabsf(c1) < 1e-30f) {
        const bool in = (q0f > -1.5f) && (q0f < n_across + 0.5f);
        a = in ? -1.0f : 1e30f;
        b = in ? (float)n_along : -1e30f;
    } else {
        const float t0 = (-1.5f - q0f) / c1, t1 = (n_across + 0.5f - q0f) / c1;
        a = fmaxf(fminf(t0, t1), -1.0f);
        b = fminf(fmaxf(t0, t1), (float)n_along);
    }
    lo = max((int)ceilf(fmaxf(a, -1.0f)), 0);
    hi = min((int)floorf(fminf(b, (float)n_along)), n_along - 1);
}

struct CandRange {
    int lo, hi;
};

// Bins whose rays can reach the axis-aligned rectangle of half-sides (hx, hy) cm centred at (xc, yc)
// in view (cs, sn): the projection of its corners (fan; the rectangle lies in front of the source)
// or of its half-width (parallel). eps absorbs float32 rounding and the rays' fixed-point
// quantisation (both far below 0.02 bins).
__device__ __forceinline__ CandRange rect_candidates(const GeomDev& g, float cs, float sn, float xc, float yc, float hx,
                                                     float hy) {
    const float eps = 0.02f;
    float kmin, kmax;
    if (g.kind == DECT_PARALLEL) {
        const float kc = fmaf(fmaf(xc, cs, yc * sn), g.inv_du, g.k0);
        const float h = fmaf(hx, fabsf(cs), hy * fabsf(sn)) * g.inv_du;
        kmin = kc - h;
        kmax = kc + h;
    } else {
        const float num = fmaf(-xc, sn, yc * cs), den = g.sod - fmaf(xc, cs, yc * sn);
        const float nx_ = -hx * sn, dx_ = -hx * cs;
        const float ny_ = hy * cs, dy_ = -hy * sn;
        const float u1 = __fdividef(num + nx_ + ny_, den + dx_ + dy_);
        const float u2 = __fdividef(num + nx_ - ny_, den + dx_ - dy_);
        const float u3 = __fdividef(num - nx_ + ny_, den - dx_ + dy_);
        const float u4 = __fdividef(num - nx_ - ny_, den - dx_ - dy_);
        kmin = fmaf(g.k1, fminf(fminf(u1, u2), fminf(u3, u4)), g.k0);
        kmax = fmaf(g.k1, fmaxf(fmaxf(u1, u2), fmaxf(u3, u4)), g.k0);
    }
    CandRange c;
    c.lo = max(0, (int)ceilf(fmaxf(kmin - eps, -1.0f)));
    c.hi = min(g.nb - 1, (int)floorf(fminf(kmax + eps, (float)g.nb)));
    return c;
}

}  // namespace dect
