// Forward projector R and its exact adjoint R^T (the projection matrix of
// Eq. 2-3; Table 1 counts their applications), for parallel and flat-detector
// fan beams.
//
// Sample positions are 32.32 fixed point. A ray is sampled once per column
// (axis 0) or row (axis 1) at position q(t) = q0 + t * slope (t the column or
// row index), so stepping is an exact 64-bit integer add: the integer part is
// the lower interpolation neighbour and the top 23 fraction bits give the
// interpolation weight by a bit-cast, without float rounding or conversions.
// Positions carry ~1e-7 pixel error against the exact geometry (float32
// positions would carry ~3e-5 near |q| = 512).
//
// R: one thread per ray; Joseph's linear interpolation between the two
// neighbours; the image is read through a pair texture (both neighbours of
// both bases in one 16-byte load).
//
// R^T: one thread per pixel, gathering over views. For each view it bounds
// the detector interval that can reach the pixel (the projection of the
// 2-pixel cross around it), then evaluates each candidate ray's position at
// the pixel's column (row) with the same integers R steps through, so both
// kernels apply bit-identical interpolation weights and <R x, y> = <x, R^T y>
// holds to float32 summation rounding. No atomics: the result is
// deterministic.
#include <cuda_runtime.h>
#include <math.h>

#include "dect_internal.cuh"

namespace dect {

// ---------------------------------------------------------------------------------------------
// per-ray table, computed once per geometry in float64 and rounded to float32

__global__ void k_ray_table(dect_geom_desc d, int4* __restrict__ rays, float4* __restrict__ views) {
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
    // position at index 0 of the sampled axis and the slope, in pixel units
    double q0, slope, w;
    int axis;
    if (fabs(dx) >= fabs(dy)) {
        slope = dy / dx;
        q0 = (py - px * slope) / d.pixel_cm + 0.5 * (d.ny - 1) - 0.5 * (d.nx - 1) * slope;
        w = d.pixel_cm / fabs(dx);
        axis = 0;
    } else {
        slope = dx / dy;
        q0 = (px - py * slope) / d.pixel_cm + 0.5 * (d.nx - 1) - 0.5 * (d.ny - 1) * slope;
        w = d.pixel_cm / fabs(dy);
        axis = 1;
    }
    const long long q0_fx = llrint(q0 * 4294967296.0);        // 32.32
    const int slope_fx = (int)llrint(slope * 1073741824.0);    // 2.30, |slope| <= 1
    const float wf = (float)w;
    rays[r] = make_int4((int)(unsigned)(q0_fx & 0xffffffffll), (int)(q0_fx >> 32), slope_fx,
                        __float_as_int(axis ? -wf : wf));
    if (k == 0) views[v] = make_float4((float)c, (float)s, 0.0f, 0.0f);
}

cudaError_t build_ray_table(const dect_geom_desc& d, int4* rays, float4* views, cudaStream_t st) {
    const int64_t n = (int64_t)d.n_views * d.n_bins;
    k_ray_table<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(d, rays, views);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------------------------
// pair textures

__device__ __forceinline__ float2 img_at(const float2* __restrict__ img, int nx, int ny, int j, int i) {
    if (j < 0 || j >= ny || i < 0 || i >= nx) return make_float2(0.f, 0.f);
    return __ldg(img + (size_t)j * nx + i);
}

// TX[i][jj] from a 32 (jj) x 32 (i) tile; rows jj-2 .. jj+29 staged in shared memory.
__global__ void __launch_bounds__(256) k_texture_x(const SliceDesc* __restrict__ dsl, BlockMap map,
                                                   const float2* __restrict__ img, float4* __restrict__ tx) {
    __shared__ float2 tile[33][33];
    int local;
    const int s = slice_of(map, blockIdx.x, local);
    const SliceDesc& d = dsl[s];
    const int nx = d.g.nx, ny = d.g.ny;
    const int tiles_i = (nx + 31) / 32;
    const int jt = (local / tiles_i) * 32, it = (local % tiles_i) * 32;
    const float2* im = img + d.img_off;
    // stage rows jt-2 .. jt+30 (33 rows), columns it .. it+31
    for (int e = threadIdx.x; e < 33 * 32; e += blockDim.x) {
        const int rr = e / 32, cc = e % 32;
        tile[rr][cc] = img_at(im, nx, ny, jt - 2 + rr, it + cc);
    }
    __syncthreads();
    float4* out = tx + d.tx_off;
    const int ld = ny + 3;
    for (int e = threadIdx.x; e < 32 * 32; e += blockDim.x) {
        const int ci = e / 32, cj = e % 32;  // consecutive threads walk jj: coalesced stores
        const int i = it + ci, jj = jt + cj;
        if (i < nx && jj < ld) {
            const float2 a = tile[cj][ci], b = tile[cj + 1][ci];
            out[(size_t)i * ld + jj] = make_float4(a.x, a.y, b.x, b.y);
        }
    }
}

// TY[j][ii], one entry per thread.
__global__ void __launch_bounds__(256) k_texture_y(const SliceDesc* __restrict__ dsl, BlockMap map,
                                                   const float2* __restrict__ img, float4* __restrict__ ty) {
    int local;
    const int s = slice_of(map, blockIdx.x, local);
    const SliceDesc& d = dsl[s];
    const int nx = d.g.nx, ny = d.g.ny, ld = nx + 3;
    const int64_t e = (int64_t)local * blockDim.x + threadIdx.x;
    if (e >= (int64_t)ny * ld) return;
    const int j = (int)(e / ld), ii = (int)(e % ld);
    const float2* im = img + d.img_off;
    const float2 a = img_at(im, nx, ny, j, ii - 2), b = img_at(im, nx, ny, j, ii - 1);
    ty[d.ty_off + e] = make_float4(a.x, a.y, b.x, b.y);
}

static int tx_blocks(int nx, int ny) { return ((nx + 31) / 32) * ((ny + 3 + 31) / 32); }
static int ty_blocks(int nx, int ny) { return (int)(((int64_t)ny * (nx + 3) + 255) / 256); }

// Textures of the batched solver: two maps (TX tiles, TY blocks).
void launch_textures(const SliceDesc* dsl, const BlockMap& mx, int nbx, const BlockMap& my, int nby,
                     const float2* img, float4* tx, float4* ty, cudaStream_t st) {
    k_texture_x<<<nbx, 256, 0, st>>>(dsl, mx, img, tx);
    k_texture_y<<<nby, 256, 0, st>>>(dsl, my, img, ty);
}

// planar input (1 or 2 channels) -> interleaved float2 image
__global__ void k_pack_planar(const float* __restrict__ in, int nch, int64_t n, float2* __restrict__ out) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    out[e] = make_float2(__ldg(in + e), nch > 1 ? __ldg(in + n + e) : 0.0f);
}

// ---------------------------------------------------------------------------------------------
// forward projector

// Fixed-point helpers: a ray entry is {q0 low word, q0 high word, slope * 2^30, +-w} with the sign of
// w giving the axis (negative: sampled per row).
__device__ __forceinline__ long long ray_q0(const int4 P) {
    return ((long long)P.y << 32) | (long long)(unsigned)P.x;
}
__device__ __forceinline__ long long ray_step(const int4 P) { return (long long)P.z << 2; }
__device__ __forceinline__ bool ray_axis(const int4 P) { return P.w < 0; }
__device__ __forceinline__ float ray_w(const int4 P) { return fabsf(__int_as_float(P.w)); }
// interpolation weight of the upper neighbour: the top 23 fraction bits as a float in [0, 1)
__device__ __forceinline__ float frac_of(long long q) {
    return __uint_as_float(0x3f800000u | ((unsigned)q >> 9)) - 1.0f;
}

// Index range [lo, hi] along the sampled axis whose positions lie in [-1.5, n_across + 0.5): it
// contains every sample with a non-zero weight (positions in (-1, n_across)) and keeps the lower
// neighbour in [-2, n_across]. Float estimate; the 0.5-pixel margins absorb its rounding.
__device__ __forceinline__ void sample_range(const int4 P, int n_along, int n_across, int& lo, int& hi) {
    const float q0 = (float)P.y * 4294967296.0f + (float)(unsigned)P.x;
    const float q0f = q0 * 2.3283064365386963e-10f;  // 2^-32
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

// Sum over the ray's samples of the interpolated {c, p}; returns unweighted sums.
__device__ __forceinline__ float2 ray_sum(const int4 P, const GeomDev& g, const float4* __restrict__ tx,
                                          const float4* __restrict__ ty) {
    float ac = 0.f, ap = 0.f;
    const bool ax = ray_axis(P);
    const int n_along = ax ? g.ny : g.nx, n_across = ax ? g.nx : g.ny;
    const float4* tex = ax ? ty : tx;
    const int ld = n_across + 3;
    int lo, hi;
    sample_range(P, n_along, n_across, lo, hi);
    const long long step = ray_step(P);
    long long q = ray_q0(P) + (long long)lo * step;
    const float4* row = tex + (size_t)lo * ld;
    for (int t = lo; t <= hi; ++t, q += step, row += ld) {
        const int jj = min(max((int)(q >> 32) + 2, 0), n_across + 2);
        const float f = frac_of(q);
        const float4 v = __ldg(row + jj);
        ac += fmaf(f, v.z - v.x, v.x);
        ap += fmaf(f, v.w - v.y, v.y);
    }
    return make_float2(ac, ap);
}

__global__ void __launch_bounds__(kRaysPerBlock) k_project(const SliceDesc* __restrict__ dsl, BlockMap map,
                                                           const float4* __restrict__ tx,
                                                           const float4* __restrict__ ty, float2* __restrict__ out) {
    int local;
    const int s = slice_of(map, blockIdx.x, local);
    const SliceDesc& d = dsl[s];
    const int64_t r = (int64_t)local * kRaysPerBlock + threadIdx.x;
    if (r >= (int64_t)d.g.nv * d.g.nb) return;
    const int4 P = __ldg(d.g.rays + r);
    const float2 acc = ray_sum(P, d.g, tx + d.tx_off, ty + d.ty_off);
    const float w = ray_w(P);
    out[d.sino_off + r] = make_float2(w * acc.x, w * acc.y);
}

__global__ void __launch_bounds__(kRaysPerBlock) k_project_planar(SliceDesc d, const float4* __restrict__ tx,
                                                                  const float4* __restrict__ ty,
                                                                  float* __restrict__ out, int nch) {
    const int64_t n = (int64_t)d.g.nv * d.g.nb;
    const int64_t r = (int64_t)blockIdx.x * kRaysPerBlock + threadIdx.x;
    if (r >= n) return;
    const int4 P = __ldg(d.g.rays + r);
    const float2 acc = ray_sum(P, d.g, tx, ty);
    const float w = ray_w(P);
    out[r] = w * acc.x;
    if (nch > 1) out[n + r] = w * acc.y;
}

void launch_project(const SliceDesc* dsl, const BlockMap& map, int nblk, const float4* tx, const float4* ty,
                    float2* out, cudaStream_t st) {
    k_project<<<nblk, kRaysPerBlock, 0, st>>>(dsl, map, tx, ty, out);
}

// ---------------------------------------------------------------------------------------------
// gathering backprojector

struct CandRange {
    int lo, hi;
};

// Bins whose rays can have a non-zero weight at pixel centre (x, y) (cm) in view (cs, sn).
__device__ __forceinline__ CandRange candidates(const GeomDev& g, float cs, float sn, float x, float y) {
    const float eps = 0.02f;
    const float half_nb = 0.5f * (g.nb - 1);
    float kmin, kmax;
    if (g.kind == DECT_PARALLEL) {
        const float uc = fmaf(x, cs, y * sn);
        const float h = g.pix * fmaxf(fabsf(cs), fabsf(sn));
        kmin = (uc - h - g.uoff) / g.du + half_nb;
        kmax = (uc + h - g.uoff) / g.du + half_nb;
    } else {
        // u(P) = sdd (P . e) / (sod - P . n), e = (-sin, cos), n = (cos, sin); the pixel's
        // interpolation support is the cross {x} x (y-pix, y+pix) U (x-pix, x+pix) x {y}
        const float num = fmaf(-x, sn, y * cs);
        const float den = g.sod - fmaf(x, cs, y * sn);
        const float dc = g.pix * cs, ds = g.pix * sn;
        const float u1 = __fdividef(num + dc, den - ds);
        const float u2 = __fdividef(num - dc, den + ds);
        const float u3 = __fdividef(num - ds, den - dc);
        const float u4 = __fdividef(num + ds, den + dc);
        const float umin = g.sdd * fminf(fminf(u1, u2), fminf(u3, u4));
        const float umax = g.sdd * fmaxf(fmaxf(u1, u2), fmaxf(u3, u4));
        kmin = (umin - g.uoff) / g.du + half_nb;
        kmax = (umax - g.uoff) / g.du + half_nb;
    }
    CandRange c;
    c.lo = max(0, (int)ceilf(fmaxf(kmin - eps, -1.0f)));
    c.hi = min(g.nb - 1, (int)floorf(fminf(kmax + eps, (float)g.nb)));
    return c;
}

// Weight with which ray P samples pixel (i, j) (without the ray's w): the same integers as ray_sum.
__device__ __forceinline__ float pixel_weight(const int4 P, int i, int j) {
    const bool ax = ray_axis(P);
    const int t = ax ? j : i, across = ax ? i : j;
    const long long q = ray_q0(P) + (long long)t * ray_step(P);
    const int q0 = (int)(q >> 32);
    const float f = frac_of(q);
    return q0 == across ? 1.0f - f : (q0 + 1 == across ? f : 0.0f);
}

__device__ __forceinline__ float2 gather_pixel(const GeomDev& g, const float2* __restrict__ sino, int i, int j) {
    const float x = ((float)i - g.cx) * g.pix, y = ((float)j - g.cy) * g.pix;
    float ac = 0.f, ap = 0.f;
    for (int v = 0; v < g.nv; ++v) {
        const float4 V = __ldg(g.views + v);
        const CandRange cr = candidates(g, V.x, V.y, x, y);
        const int4* rv = g.rays + (size_t)v * g.nb;
        const float2* sv = sino + (size_t)v * g.nb;
        for (int k = cr.lo; k <= cr.hi; ++k) {
            const int4 P = __ldg(rv + k);
            const float wgt = pixel_weight(P, i, j);
            if (wgt != 0.0f) {
                const float2 sv2 = __ldg(sv + k);
                const float ww = ray_w(P) * wgt;
                ac = fmaf(ww, sv2.x, ac);
                ap = fmaf(ww, sv2.y, ap);
            }
        }
    }
    return make_float2(ac, ap);
}

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

template <int MODE>
__global__ void __launch_bounds__(kBpTile * kBpTile) k_backproject(const SliceDesc* __restrict__ dsl, BlockMap map,
                                                                   const float2* __restrict__ sino,
                                                                   float2* __restrict__ out, BpEpilogue ep) {
    int local;
    const int s = slice_of(map, blockIdx.x, local);
    const SliceDesc& d = dsl[s];
    const int nx = d.g.nx, ny = d.g.ny;
    const int tiles_x = (nx + kBpTile - 1) / kBpTile;
    const int i = (local % tiles_x) * kBpTile + (threadIdx.x % kBpTile);
    const int j = (local / tiles_x) * kBpTile + (threadIdx.x / kBpTile);
    const bool valid = (i < nx) && (j < ny);
    float2 acc = make_float2(0.f, 0.f);
    if (valid) acc = gather_pixel(d.g, sino + d.sino_off, i, j);
    double dot_c = 0.0, dot_p = 0.0;
    if (valid) {
        const int64_t off = d.img_off;
        const size_t e = (size_t)j * nx + i;
        float2 r = acc;
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
            dot_c = (double)pc.x * (double)r.x;
            dot_p = (double)pc.y * (double)r.y;
        }
        out[off + e] = r;
    }
    if (MODE == BP_AP || MODE == BP_AP_NOGRAD) {
        // deterministic block reduction of the two partial dot products
        __shared__ double red[2][kBpTile * kBpTile / 32];
        for (int o = 16; o > 0; o >>= 1) {
            dot_c += __shfl_down_sync(0xffffffffu, dot_c, o);
            dot_p += __shfl_down_sync(0xffffffffu, dot_p, o);
        }
        const int w = threadIdx.x / 32, l = threadIdx.x % 32;
        if (l == 0) {
            red[0][w] = dot_c;
            red[1][w] = dot_p;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            double sc = 0.0, sp = 0.0;
            for (int q = 0; q < kBpTile * kBpTile / 32; ++q) {
                sc += red[0][q];
                sp += red[1][q];
            }
            ep.partial[2 * (size_t)blockIdx.x] = sc;
            ep.partial[2 * (size_t)blockIdx.x + 1] = sp;
        }
    }
}

__global__ void __launch_bounds__(kBpTile * kBpTile) k_backproject_planar(SliceDesc d, const float2* __restrict__ sino,
                                                                          float* __restrict__ out, int nch) {
    const int nx = d.g.nx, ny = d.g.ny;
    const int tiles_x = (nx + kBpTile - 1) / kBpTile;
    const int i = (blockIdx.x % tiles_x) * kBpTile + (threadIdx.x % kBpTile);
    const int j = (blockIdx.x / tiles_x) * kBpTile + (threadIdx.x / kBpTile);
    if (i >= nx || j >= ny) return;
    const float2 acc = gather_pixel(d.g, sino, i, j);
    const size_t e = (size_t)j * nx + i;
    out[e] = acc.x;
    if (nch > 1) out[(size_t)nx * ny + e] = acc.y;
}

int bp_tiles(int nx, int ny) { return ((nx + kBpTile - 1) / kBpTile) * ((ny + kBpTile - 1) / kBpTile); }

void launch_backproject(int mode, const SliceDesc* dsl, const BlockMap& map, int nblk, const float2* sino,
                        float2* out, const BpEpilogue& ep, cudaStream_t st) {
    const int T = kBpTile * kBpTile;
    switch (mode) {
        case BP_PLAIN: k_backproject<BP_PLAIN><<<nblk, T, 0, st>>>(dsl, map, sino, out, ep); break;
        case BP_R0: k_backproject<BP_R0><<<nblk, T, 0, st>>>(dsl, map, sino, out, ep); break;
        case BP_AP: k_backproject<BP_AP><<<nblk, T, 0, st>>>(dsl, map, sino, out, ep); break;
        case BP_R0_NOGRAD: k_backproject<BP_R0_NOGRAD><<<nblk, T, 0, st>>>(dsl, map, sino, out, ep); break;
        case BP_AP_NOGRAD: k_backproject<BP_AP_NOGRAD><<<nblk, T, 0, st>>>(dsl, map, sino, out, ep); break;
        default: break;
    }
}

// ---------------------------------------------------------------------------------------------
// single-slice planar entry points (dect_project / dect_backproject)

__global__ void k_texture_x_single(SliceDesc d, const float2* __restrict__ img, float4* __restrict__ tx) {
    // same as k_texture_x for one slice without a block map
    __shared__ float2 tile[33][33];
    const int nx = d.g.nx, ny = d.g.ny;
    const int tiles_i = (nx + 31) / 32;
    const int jt = (blockIdx.x / tiles_i) * 32, it = (blockIdx.x % tiles_i) * 32;
    for (int e = threadIdx.x; e < 33 * 32; e += blockDim.x) {
        const int rr = e / 32, cc = e % 32;
        tile[rr][cc] = img_at(img, nx, ny, jt - 2 + rr, it + cc);
    }
    __syncthreads();
    const int ld = ny + 3;
    for (int e = threadIdx.x; e < 32 * 32; e += blockDim.x) {
        const int ci = e / 32, cj = e % 32;
        const int i = it + ci, jj = jt + cj;
        if (i < nx && jj < ld) {
            const float2 a = tile[cj][ci], b = tile[cj + 1][ci];
            tx[(size_t)i * ld + jj] = make_float4(a.x, a.y, b.x, b.y);
        }
    }
}

__global__ void k_texture_y_single(SliceDesc d, const float2* __restrict__ img, float4* __restrict__ ty) {
    const int nx = d.g.nx, ny = d.g.ny, ld = nx + 3;
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (int64_t)ny * ld) return;
    const int j = (int)(e / ld), ii = (int)(e % ld);
    const float2 a = img_at(img, nx, ny, j, ii - 2), b = img_at(img, nx, ny, j, ii - 1);
    ty[e] = make_float4(a.x, a.y, b.x, b.y);
}

// `scratch` must hold nx*ny float2
void project_single(const SliceDesc& sd, const float* img, int nch, float2* scratch, float4* tx, float4* ty,
                    float* out, cudaStream_t st) {
    const int64_t np = (int64_t)sd.g.nx * sd.g.ny;
    k_pack_planar<<<(unsigned)((np + 255) / 256), 256, 0, st>>>(img, nch, np, scratch);
    k_texture_x_single<<<tx_blocks(sd.g.nx, sd.g.ny), 256, 0, st>>>(sd, scratch, tx);
    k_texture_y_single<<<ty_blocks(sd.g.nx, sd.g.ny), 256, 0, st>>>(sd, scratch, ty);
    const int64_t nr = (int64_t)sd.g.nv * sd.g.nb;
    k_project_planar<<<(unsigned)((nr + kRaysPerBlock - 1) / kRaysPerBlock), kRaysPerBlock, 0, st>>>(sd, tx, ty, out,
                                                                                                      nch);
}

// `packed` must hold nv*nb float2
void backproject_single(const SliceDesc& sd, const float* sino, int nch, float2* packed, float* out,
                        cudaStream_t st) {
    const int64_t nr = (int64_t)sd.g.nv * sd.g.nb;
    k_pack_planar<<<(unsigned)((nr + 255) / 256), 256, 0, st>>>(sino, nch, nr, packed);
    k_backproject_planar<<<bp_tiles(sd.g.nx, sd.g.ny), kBpTile * kBpTile, 0, st>>>(sd, packed, out, nch);
}

int texture_x_blocks(int nx, int ny) { return tx_blocks(nx, ny); }
int texture_y_blocks(int nx, int ny) { return ty_blocks(nx, ny); }

}  // namespace dect
