// Per-pixel epilogues of the backprojector: the CG pieces of Eq. 12 that are computed
// where R^T's result for a pixel is produced (r0 = R^T b + D^T(y + u^y - D x) + (z + u^z - x), and
// A p = R^T q + D^T D p + p with the partial sums of <p, A p>), shared by the backprojector kernels.
#pragma once

#include <cuda_runtime.h>

#include "dect_internal.cuh"
#include "reduce.cuh"

namespace dect {

__device__ __forceinline__ float2 f2(const float2* __restrict__ a, int nx, int ny, int j, int i) {
    return (i < 0 || i >= nx || j < 0 || j >= ny) ? make_float2(0.f, 0.f) : __ldg(a + (size_t)j * nx + i);
}

// forward differences of a float2 image at (j, i): {dx_c, dy_c, dx_p, dy_p}, 0 at the last column/row
__device__ __forceinline__ float4 grad_at(const float2* __restrict__ a, int nx, int ny, int j, int i) {
    const float2 c = __ldg(a + (size_t)j * nx + i);
    float4 g = make_float4(0.f, 0.f, 0.f, 0.f);
    if (i < nx - 1) {
        const float2 r = __ldg(a + (size_t)j * nx + i + 1);
        g.x = r.x - c.x;
        g.z = r.y - c.y;
    }
    if (j < ny - 1) {
        const float2 u = __ldg(a + (size_t)(j + 1) * nx + i);
        g.y = u.x - c.x;
        g.w = u.y - c.y;
    }
    return g;
}

// (D^T t)(j, i) for a field t given at (j, i), (j, i-1) and (j-1, i): only components whose
// D row is non-zero (x-component at i < nx-1, y-component at j < ny-1) take part.
__device__ __forceinline__ float2 div_t(float4 t_ij, float4 t_im, float4 t_jm, int nx, int ny, int j, int i) {
    float c = 0.f, p = 0.f;
    if (i < nx - 1) { c -= t_ij.x; p -= t_ij.z; }
    if (i >= 1) { c += t_im.x; p += t_im.z; }
    if (j < ny - 1) { c -= t_ij.y; p -= t_ij.w; }
    if (j >= 1) { c += t_jm.y; p += t_jm.w; }
    return make_float2(c, p);
}

__device__ __forceinline__ float4 y_plus_u_minus_grad(const BpEpilogue& ep, int64_t off, int nx, int ny, int j, int i) {
    const float2* x = ep.x + off;
    const size_t e = (size_t)j * nx + i;
    const float4 y = __ldg(ep.y + off + e), u = __ldg(ep.uy + off + e);
    const float4 g = grad_at(x, nx, ny, j, i);
    return make_float4(y.x + u.x - g.x, y.y + u.y - g.y, y.z + u.z - g.z, y.w + u.w - g.w);
}

__device__ __forceinline__ float4 grad_of(const float2* __restrict__ p, int nx, int ny, int j, int i) {
    return grad_at(p, nx, ny, j, i);
}

// Finishes pixel (i, j) of slice d from its backprojected value r (both bases): adds the mode's
// image-domain terms, accumulates <p, A p> (AP modes) and stores to `out` (interleaved, at the
// slice's offset) or to `planar` ([nch][ny][nx], single slice).
template <int MODE>
__device__ __forceinline__ void bp_pixel_epilogue(const SliceDesc& d, int i, int j, float2 r, const BpEpilogue& ep,
                                                  float2* __restrict__ out, float* __restrict__ planar, int nch,
                                                  float& dot_c, float& dot_p) {
    const int nx = d.g.nx, ny = d.g.ny;
    const int64_t off = d.img_off;
    const size_t e = (size_t)j * nx + i;
    if (MODE == BP_R0 || MODE == BP_R0_NOGRAD) {
        const float2 xc = __ldg(ep.x + off + e), z = __ldg(ep.z + off + e), uz = __ldg(ep.uz + off + e);
        r.x += z.x + uz.x - xc.x;
        r.y += z.y + uz.y - xc.y;
        if (MODE == BP_R0) {
            const float4 t_ij = y_plus_u_minus_grad(ep, off, nx, ny, j, i);
            const float4 t_im = i >= 1 ? y_plus_u_minus_grad(ep, off, nx, ny, j, i - 1) : make_float4(0, 0, 0, 0);
            const float4 t_jm = j >= 1 ? y_plus_u_minus_grad(ep, off, nx, ny, j - 1, i) : make_float4(0, 0, 0, 0);
            const float2 dt = div_t(t_ij, t_im, t_jm, nx, ny, j, i);
            r.x += dt.x;
            r.y += dt.y;
        }
    } else if (MODE == BP_AP || MODE == BP_AP_NOGRAD) {
        const float2* p = ep.p + off;
        const float2 pc = __ldg(p + e);
        r.x += pc.x;
        r.y += pc.y;
        if (MODE == BP_AP) {
            const float4 g_ij = grad_of(p, nx, ny, j, i);
            const float4 g_im = i >= 1 ? grad_of(p, nx, ny, j, i - 1) : make_float4(0, 0, 0, 0);
            const float4 g_jm = j >= 1 ? grad_of(p, nx, ny, j - 1, i) : make_float4(0, 0, 0, 0);
            const float2 dt = div_t(g_ij, g_im, g_jm, nx, ny, j, i);
            r.x += dt.x;
            r.y += dt.y;
        }
        dot_c = fmaf(pc.x, r.x, dot_c);
        dot_p = fmaf(pc.y, r.y, dot_p);
    }
    if (planar) {
        planar[e] = r.x;
        if (nch > 1) planar[(size_t)nx * ny + e] = r.y;
    } else {
        out[off + e] = r;
    }
}

// Deterministic block reduction of the partial <p, A p> sums into partial[2 * blockIdx.x + {0, 1}]
// (float within a warp, float64 across warps).
__device__ __forceinline__ void bp_block_dots(float dot_c, float dot_p, double* __restrict__ partial) {
    float v[2] = {dot_c, dot_p};
    block_partials<2>(v, partial);
}

}  // namespace dect
