// Float64 forward projector R and adjoint R^T (Eq. 2-3's projection matrix) for the
// public entry points (dect_project / dect_backproject with DECT_F64), used where a float64 result
// is wanted, e.g. gradient checks through the autograd wrappers.
//
// The float32 kernels quantise sample positions to 2^-30 pixel with a 2^-30 slope, which bounds
// their weights to ~1e-7; here every ray's position at index 0, slope and weight come from a
// float64 table built once per geometry, and both kernels evaluate a sample's position with the
// same explicit fused multiply-add, so R and R^T apply identical float64 weights. Same Joseph
// interpolation and conventions as the float32 path; simple thread-per-ray / thread-per-pixel
// kernels (float64 throughput on this GPU is low; these are not on the solver's path).
#include <cuda_runtime.h>
#include <math.h>

#include "dect_internal.cuh"
#include "ray_fixed.cuh"

namespace dect {

// {position at index 0 of the sampled axis, slope, weight, axis (0: per column, 1: per row)}
__global__ void k_ray_table_f64(dect_geom_desc d, double4_32a* __restrict__ rays) {
    const int64_t n = (int64_t)d.n_views * d.n_bins;
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    const int v = (int)(r / d.n_bins), k = (int)(r % d.n_bins);
    const double th = d.angle0_rad + v * (d.angle_span_rad / d.n_views);
    double s, c;
    sincos(th, &s, &c);
    const double u = (k - 0.5 * (d.n_bins - 1)) * d.bin_pitch_cm + d.bin_offset_cm;
    double px, py, dx, dy;
    if (d.kind == DECT_PARALLEL) {
        px = u * c;
        py = u * s;
        dx = -s;
        dy = c;
    } else {
        const double sx = d.sod_cm * c, sy = d.sod_cm * s;
        const double qx = -(d.sdd_cm - d.sod_cm) * c - u * s;
        const double qy = -(d.sdd_cm - d.sod_cm) * s + u * c;
        const double ex = qx - sx, ey = qy - sy;
        const double len = sqrt(ex * ex + ey * ey);
        px = sx;
        py = sy;
        dx = ex / len;
        dy = ey / len;
    }
    if (fabs(dx) >= fabs(dy)) {
        const double slope = dy / dx;
        rays[r] = make_double4_32a((py - px * slope) / d.pixel_cm + 0.5 * (d.ny - 1) - 0.5 * (d.nx - 1) * slope, slope,
                               d.pixel_cm / fabs(dx), 0.0);
    } else {
        const double slope = dx / dy;
        rays[r] = make_double4_32a((px - py * slope) / d.pixel_cm + 0.5 * (d.nx - 1) - 0.5 * (d.ny - 1) * slope, slope,
                               d.pixel_cm / fabs(dy), 1.0);
    }
}

cudaError_t build_ray_table_f64(const dect_geom_desc& d, double4_32a* rays, cudaStream_t st) {
    const int64_t n = (int64_t)d.n_views * d.n_bins;
    k_ray_table_f64<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(d, rays);
    return cudaGetLastError();
}

__device__ __forceinline__ double img64(const double* __restrict__ im, int nx, int ny, int j, int i) {
    return (i < 0 || i >= nx || j < 0 || j >= ny) ? 0.0 : __ldg(im + (size_t)j * nx + i);
}

// out[c][ray] = R x[c], planar float64
__global__ void k_project_f64(GeomDev g, const double4_32a* __restrict__ rays, const double* __restrict__ x, int nch,
                              double* __restrict__ out) {
    const int64_t n = (int64_t)g.nv * g.nb;
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    const double4_32a P = rays[r];
    const bool ax = P.w != 0.0;
    const int n_along = ax ? g.ny : g.nx, n_across = ax ? g.nx : g.ny;
    // indices whose positions lie in (-1, n_across): the only ones with a non-zero weight
    int lo = 0, hi = n_along - 1;
    if (P.y != 0.0) {
        const double t0 = (-1.0 - P.x) / P.y, t1 = ((double)n_across - P.x) / P.y;
        lo = max(lo, (int)floor(fmax(fmin(t0, t1), -1.0)));
        hi = min(hi, (int)ceil(fmin(fmax(t0, t1), (double)n_along)));
    } else if (!(P.x > -1.0 && P.x < n_across)) {
        hi = -1;
    }
    const size_t plane = (size_t)g.nx * g.ny;
    for (int c = 0; c < nch; ++c) {
        const double* im = x + c * plane;
        double acc = 0.0;
        for (int t = lo; t <= hi; ++t) {
            const double q = __fma_rn((double)t, P.y, P.x);
            const double fl = floor(q);
            const double f = q - fl;
            const int h = (int)fl;
            const double a = ax ? img64(im, g.nx, g.ny, t, h) : img64(im, g.nx, g.ny, h, t);
            const double b = ax ? img64(im, g.nx, g.ny, t, h + 1) : img64(im, g.nx, g.ny, h + 1, t);
            acc += (1.0 - f) * a + f * b;
        }
        out[c * n + r] = P.z * acc;
    }
}

// x[c][pixel] = R^T s[c]: gathers per pixel over views and candidate bins
__global__ void k_backproject_f64(GeomDev g, const double4_32a* __restrict__ rays, const double* __restrict__ sino, int nch,
                                  double* __restrict__ out) {
    const int64_t np = (int64_t)g.nx * g.ny;
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= np) return;
    const int j = (int)(e / g.nx), i = (int)(e % g.nx);
    // rays with a non-zero weight at (i, j) pass within 1 pixel of it: candidates of the square of
    // half-side 1.5 pixels around the 2x2 block with top-left (i, j)
    const float xc = ((float)i + 0.5f - g.cx) * g.pix, yc = ((float)j + 0.5f - g.cy) * g.pix;
    const int64_t n = (int64_t)g.nv * g.nb;
    double acc0 = 0.0, acc1 = 0.0;
    for (int v = 0; v < g.nv; ++v) {
        const float4 V = __ldg(g.views + v);
        const CandRange cr = rect_candidates(g, V.x, V.y, xc, yc, 1.5f * g.pix, 1.5f * g.pix);
        for (int k = cr.lo; k <= cr.hi; ++k) {
            const int64_t r = (int64_t)v * g.nb + k;
            const double4_32a P = rays[r];
            const bool ax = P.w != 0.0;
            const int t = ax ? j : i, across = ax ? i : j;
            const double q = __fma_rn((double)t, P.y, P.x);
            const double fl = floor(q);
            const double f = q - fl;
            const int h = (int)fl;
            const double wgt = h == across ? 1.0 - f : (h + 1 == across ? f : 0.0);
            if (wgt != 0.0) {
                acc0 += P.z * wgt * sino[r];
                if (nch > 1) acc1 += P.z * wgt * sino[n + r];
            }
        }
    }
    out[e] = acc0;
    if (nch > 1) out[np + e] = acc1;
}

void project_single_f64(const GeomDev& g, const double4_32a* rays, const double* x, int nch, double* out,
                        cudaStream_t st) {
    const int64_t n = (int64_t)g.nv * g.nb;
    k_project_f64<<<(unsigned)((n + 127) / 128), 128, 0, st>>>(g, rays, x, nch, out);
}

void backproject_single_f64(const GeomDev& g, const double4_32a* rays, const double* sino, int nch, double* out,
                            cudaStream_t st) {
    const int64_t np = (int64_t)g.nx * g.ny;
    k_backproject_f64<<<(unsigned)((np + 127) / 128), 128, 0, st>>>(g, rays, sino, nch, out);
}

}  // namespace dect
