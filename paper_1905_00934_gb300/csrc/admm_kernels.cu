// Element-wise and reduction kernels of one ADMM iteration (Sec. 3.2-3.3):
// the CG vector updates and scalars of Eq. 12, the TV shrinkage and
// non-negativity updates (Eq. 9-10), the dual update (Eq. 11) with the
// residual sums, residual-balancing rho, and the state (re)initialisation.
//
// Reductions are deterministic: each block writes its partial sums (float64)
// to a slot indexed by its block number, and one block per slice adds its
// slots in a fixed order. All scalars stay on the device.
#include <cuda_runtime.h>

#include <algorithm>
#include <math.h>

#include "admm_kernels.cuh"
#include "prec.cuh"
#include "reduce.cuh"

namespace dect {

// ---- Eq. 12 pieces ------------------------------------------------------------------------------

// b = a + u^a - R x (the sinogram part of the CG residual)
template <class S2>
__global__ void __launch_bounds__(256) k_sino_resid(const SliceDesc* __restrict__ dsl, BlockMap map,
                                                    const S2* __restrict__ a, const S2* __restrict__ ua,
                                                    const S2* __restrict__ Rx, S2* __restrict__ b) {
    int local;
    const int s = slice_of(map, blockIdx.x, local);
    const SliceDesc& d = dsl[s];
    const int64_t r = (int64_t)local * 256 + threadIdx.x;
    if (r >= (int64_t)d.g.nv * d.g.nb) return;
    const int64_t e = d.sino_off + r;
    const float2 av = ldg2(a + e), uv = ldg2(ua + e), rv = ldg2(Rx + e);
    st2(b + e, make_float2(av.x + uv.x - rv.x, av.y + uv.y - rv.y));
}

// rs = <r, M^-1 r> from the preconditioner's row partials; after the first CG step also beta
__global__ void __launch_bounds__(256) k_rs_reduce(const double* __restrict__ part, const int* __restrict__ rows_prefix,
                                                   SliceScalars* __restrict__ sc, int first) {
    const int s = blockIdx.x;
    double v[2];
    slice_sum<2>(part, rows_prefix, s, v);
    if (threadIdx.x == 0) {
        for (int c = 0; c < 2; ++c) {
            if (!first) sc[s].beta[c] = sc[s].rs[c] > 0.0 ? v[c] / sc[s].rs[c] : 0.0;
            sc[s].beta_f[c] = (float)sc[s].beta[c];
            sc[s].rs[c] = v[c];
        }
    }
}

// alpha = rs / <p, A p>
__global__ void __launch_bounds__(256) k_alpha(const double* __restrict__ part, const int* __restrict__ bp_prefix,
                                               SliceScalars* __restrict__ sc) {
    const int s = blockIdx.x;
    double v[2];
    slice_sum<2>(part, bp_prefix, s, v);
    if (threadIdx.x == 0) {
        for (int c = 0; c < 2; ++c) {
            sc[s].pAp[c] = v[c];
            sc[s].alpha[c] = v[c] > 0.0 ? sc[s].rs[c] / v[c] : 0.0;
            sc[s].alpha_f[c] = (float)sc[s].alpha[c];
        }
    }
}

// x += alpha p, r -= alpha A p (unless last) over the image blocks; R x += alpha q over the ray blocks
template <class S2>
__global__ void __launch_bounds__(256) k_cg_update(const SliceDesc* __restrict__ dsl, BlockMap pix, int nblk_pix,
                                                   BlockMap rays, const SliceScalars* __restrict__ sc,
                                                   float2* __restrict__ x, const float2* __restrict__ p,
                                                   float2* __restrict__ r, const float2* __restrict__ Ap,
                                                   S2* __restrict__ Rx, const S2* __restrict__ q, int last) {
    int local;
    const bool img = (int)blockIdx.x < nblk_pix;
    const int sb = img ? slice_of(pix, blockIdx.x, local) : slice_of(rays, blockIdx.x - nblk_pix, local);
    const float2 al = make_float2(sc[sb].alpha_f[0], sc[sb].alpha_f[1]);
    if (img) {
        const int s = sb;
        const SliceDesc& d = dsl[s];
        const int64_t k = (int64_t)local * 256 + threadIdx.x;
        if (k >= (int64_t)d.g.nx * d.g.ny) return;
        const float ac = al.x, ap = al.y;
        const int64_t e = d.img_off + k;
        // loads before stores (independent addresses; keeps them all in flight together)
        const float2 pv = __ldg(p + e);
        float2 xv = x[e];
        float2 av = make_float2(0.f, 0.f), rv = make_float2(0.f, 0.f);
        if (!last) {
            av = __ldg(Ap + e);
            rv = r[e];
        }
        xv.x = fmaf(ac, pv.x, xv.x);
        xv.y = fmaf(ap, pv.y, xv.y);
        x[e] = xv;
        if (!last) {
            rv.x = fmaf(-ac, av.x, rv.x);
            rv.y = fmaf(-ap, av.y, rv.y);
            r[e] = rv;
        }
    } else {
        const int s = sb;
        const SliceDesc& d = dsl[s];
        const int64_t k = (int64_t)local * 256 + threadIdx.x;
        if (k >= (int64_t)d.g.nv * d.g.nb) return;
        const float ac = al.x, ap = al.y;
        const int64_t e = d.sino_off + k;
        const float2 qv = ldg2(q + e);
        float2 rx = ld2(Rx + e);
        rx.x = fmaf(ac, qv.x, rx.x);
        rx.y = fmaf(ap, qv.y, rx.y);
        st2(Rx + e, rx);
    }
}

// p = s + beta p
__global__ void __launch_bounds__(256) k_cg_p(const SliceDesc* __restrict__ dsl, BlockMap pix,
                                              const SliceScalars* __restrict__ sc, const float2* __restrict__ sv,
                                              float2* __restrict__ p) {
    int local;
    const int s = slice_of(pix, blockIdx.x, local);
    const float2 be = make_float2(sc[s].beta_f[0], sc[s].beta_f[1]);
    const SliceDesc& d = dsl[s];
    const int64_t k = (int64_t)local * 256 + threadIdx.x;
    if (k >= (int64_t)d.g.nx * d.g.ny) return;
    const int64_t e = d.img_off + k;
    const float bc = be.x, bp = be.y;
    const float2 a = __ldg(sv + e);
    float2 pv = p[e];
    pv.x = fmaf(bc, pv.x, a.x);
    pv.y = fmaf(bp, pv.y, a.y);
    p[e] = pv;
}

// ---- Eq. 9-11 on the image side -----------------------------------------------------------------

__device__ __forceinline__ float shrink(float t, float tau) {
    const float m = fabsf(t) - tau;
    return m > 0.f ? copysignf(m, t) : 0.f;
}

// y = shrinkage(Dx - u^y, lambda/rho); z = max(0, x - u^z); u^y += y - Dx; u^z += z - x.
// partial[4 blk + {0,1}] = sum (y - Dx)^2 + (z - x)^2 per basis; {2,3} = sum (y - y_old)^2 + (z - z_old)^2.
__global__ void __launch_bounds__(256) k_image_update(const SliceDesc* __restrict__ dsl, BlockMap pix,
                                                      const SliceScalars* __restrict__ sc, double lam_c,
                                                      double lam_p, const float2* __restrict__ x,
                                                      float4* __restrict__ y, float4* __restrict__ uy,
                                                      float2* __restrict__ z, float2* __restrict__ uz,
                                                      double* __restrict__ partial) {
    int local;
    const int s = slice_of(pix, blockIdx.x, local);
    const SliceDesc& d = dsl[s];
    const int nx = d.g.nx, ny = d.g.ny;
    const int64_t k = (int64_t)local * 256 + threadIdx.x;
    float acc[4] = {0.f, 0.f, 0.f, 0.f};
    const float2 tau = make_float2((float)lam_c / sc[s].rho_f[0], (float)lam_p / sc[s].rho_f[1]);  // lambda / rho
    if (k < (int64_t)nx * ny) {
        const int j = (int)(k / nx), i = (int)(k % nx);
        const float2* xs = x + d.img_off;
        const int64_t e = d.img_off + k;
        // every load first (they are independent), then the arithmetic and the stores
        const float2 xc = __ldg(xs + k);
        const float2 rr = i < nx - 1 ? __ldg(xs + k + 1) : xc;
        const float2 uu = j < ny - 1 ? __ldg(xs + k + nx) : xc;
        const float4 yo = y[e];
        float4 u = uy[e];
        const float2 zo = z[e];
        float2 w = uz[e];
        const float4 g = make_float4(rr.x - xc.x, uu.x - xc.x, rr.y - xc.y, uu.y - xc.y);
        const float tc = tau.x, tp = tau.y;
        const float4 yn = make_float4(shrink(g.x - u.x, tc), shrink(g.y - u.y, tc), shrink(g.z - u.z, tp),
                                      shrink(g.w - u.w, tp));
        u.x += yn.x - g.x;
        u.y += yn.y - g.y;
        u.z += yn.z - g.z;
        u.w += yn.w - g.w;
        y[e] = yn;
        uy[e] = u;
        const float2 zn = make_float2(fmaxf(0.f, xc.x - w.x), fmaxf(0.f, xc.y - w.y));
        w.x += zn.x - xc.x;
        w.y += zn.y - xc.y;
        z[e] = zn;
        uz[e] = w;
        const float ryx = yn.x - g.x, ryy = yn.y - g.y, rpx = yn.z - g.z, rpy = yn.w - g.w;
        const float rzc = zn.x - xc.x, rzp = zn.y - xc.y;
        acc[0] = fmaf(ryx, ryx, fmaf(ryy, ryy, rzc * rzc));
        acc[1] = fmaf(rpx, rpx, fmaf(rpy, rpy, rzp * rzp));
        const float dyx = yn.x - yo.x, dyy = yn.y - yo.y, dpx = yn.z - yo.z, dpy = yn.w - yo.w;
        const float dzc = zn.x - zo.x, dzp = zn.y - zo.y;
        acc[2] = fmaf(dyx, dyx, fmaf(dyy, dyy, dzc * dzc));
        acc[3] = fmaf(dpx, dpx, fmaf(dpy, dpy, dzp * dzp));
    }
    block_partials<4>(acc, partial);
}

// residual balancing: one block per slice
__global__ void __launch_bounds__(256) k_rho_update(const double* __restrict__ part_udm,
                                                    const int* __restrict__ rays_prefix,
                                                    const double* __restrict__ part_img,
                                                    const int* __restrict__ pix_prefix, SliceScalars* __restrict__ sc,
                                                    double mu_b, double tau) {
    const int s = blockIdx.x;
    double a[4], b[4];
    slice_sum<4>(part_udm, rays_prefix, s, a);
    slice_sum<4>(part_img, pix_prefix, s, b);
    if (threadIdx.x == 0) {
        for (int c = 0; c < 2; ++c) {
            const double rp = sqrt(a[c] + b[c]);
            const double rd = sc[s].rho[c] * sqrt(a[2 + c] + b[2 + c]);
            sc[s].r_pri[c] = rp;
            sc[s].r_dual[c] = rd;
            double f = 1.0;
            if (rp > mu_b * rd) f = tau;
            else if (rd > mu_b * rp) f = 1.0 / tau;
            sc[s].factor[c] = f;
            sc[s].rho[c] *= f;
            sc[s].rho_f[c] = (float)sc[s].rho[c];
            sc[s].ifactor_f[c] = (float)(1.0 / f);
        }
        sc[s].iteration += 1;
    }
}

// scaled duals follow rho: u /= factor (no-op when both factors are 1). G blocks per slice stride over
// the slice's pixels and rays, so a slice whose rho stayed costs its G blocks one test each.
template <class S2>
__global__ void __launch_bounds__(256) k_dual_rescale(const SliceDesc* __restrict__ dsl, int G,
                                                      const SliceScalars* __restrict__ sc, float4* __restrict__ uy,
                                                      float2* __restrict__ uz, S2* __restrict__ ua) {
    const int s = blockIdx.x / G, g = blockIdx.x % G;
    const float gc = sc[s].ifactor_f[0], gp = sc[s].ifactor_f[1];  // exactly 1, 1/tau or tau
    if (gc == 1.0f && gp == 1.0f) return;
    const SliceDesc& d = dsl[s];
    const int64_t np = (int64_t)d.g.nx * d.g.ny, nr = (int64_t)d.g.nv * d.g.nb, step = (int64_t)G * blockDim.x;
    for (int64_t k = (int64_t)g * blockDim.x + threadIdx.x; k < np; k += step) {
        const int64_t e = d.img_off + k;
        float4 u = uy[e];
        float2 w = uz[e];
        u.x *= gc;
        u.y *= gc;
        u.z *= gp;
        u.w *= gp;
        uy[e] = u;
        w.x *= gc;
        w.y *= gp;
        uz[e] = w;
    }
    for (int64_t k = (int64_t)g * blockDim.x + threadIdx.x; k < nr; k += step) {
        const int64_t e = d.sino_off + k;
        float2 u = ld2(ua + e);
        u.x *= gc;
        u.y *= gp;
        st2(ua + e, u);
    }
}

// ---- monitors -------------------------------------------------------------------------------------

// partial[4 blk + {0,1}] = sum (x - x*)^2 per basis, {2,3} = sum x*^2
__global__ void __launch_bounds__(256) k_xi_partials(const SliceDesc* __restrict__ dsl, BlockMap pix,
                                                     const float2* __restrict__ x, const float2* __restrict__ truth,
                                                     double* __restrict__ partial) {
    int local;
    const int s = slice_of(pix, blockIdx.x, local);
    const SliceDesc& d = dsl[s];
    const int64_t k = (int64_t)local * 256 + threadIdx.x;
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    if (k < (int64_t)d.g.nx * d.g.ny) {
        const int64_t e = d.img_off + k;
        const float2 xv = __ldg(x + e), tv = __ldg(truth + e);
        const double dc = (double)xv.x - tv.x, dp = (double)xv.y - tv.y;
        acc[0] = dc * dc;
        acc[1] = dp * dp;
        acc[2] = (double)tv.x * tv.x;
        acc[3] = (double)tv.y * tv.y;
    }
    block_partials<4>(acc, partial);
}

__global__ void __launch_bounds__(256) k_xi_reduce(const double* __restrict__ part, const int* __restrict__ pix_prefix,
                                                   SliceScalars* __restrict__ sc) {
    const int s = blockIdx.x;
    double v[4];
    slice_sum<4>(part, pix_prefix, s, v);
    if (threadIdx.x == 0) {
        sc[s].xi_num[0] = v[0];
        sc[s].xi_num[1] = v[1];
        sc[s].xi_den[0] = v[2];
        sc[s].xi_den[1] = v[3];
    }
}

// Eq. 4's regulariser per pixel block: partial[blk] = sum lambda_c |D x_c|_1 + lambda_p |D x_p|_1
__global__ void __launch_bounds__(256) k_objective_tv(const SliceDesc* __restrict__ dsl, BlockMap pix,
                                                      const float2* __restrict__ x, double lam_c, double lam_p,
                                                      double* __restrict__ partial) {
    int local;
    const SliceDesc& d = dsl[slice_of(pix, blockIdx.x, local)];
    const int nx = d.g.nx, ny = d.g.ny;
    const int64_t k = (int64_t)local * 256 + threadIdx.x;
    double acc[1] = {0.0};
    if (k < (int64_t)nx * ny) {
        const int j = (int)(k / nx), i = (int)(k % nx);
        const float2* xs = x + d.img_off;
        const float2 c = __ldg(xs + k);
        double tc = 0.0, tp = 0.0;
        if (i < nx - 1) {
            const float2 r = __ldg(xs + k + 1);
            tc += fabs((double)r.x - c.x);
            tp += fabs((double)r.y - c.y);
        }
        if (j < ny - 1) {
            const float2 u = __ldg(xs + k + nx);
            tc += fabs((double)u.x - c.x);
            tp += fabs((double)u.y - c.y);
        }
        acc[0] = lam_c * tc + lam_p * tp;
    }
    block_partials<1>(acc, partial);
}

// objective = sum of the slice's ray partials + pixel partials (one block per slice)
__global__ void __launch_bounds__(256) k_objective_reduce(const double* __restrict__ part_rays,
                                                          const int* __restrict__ rays_prefix,
                                                          const double* __restrict__ part_pix,
                                                          const int* __restrict__ pix_prefix,
                                                          SliceScalars* __restrict__ sc) {
    const int s = blockIdx.x;
    double a[1], b[1];
    slice_sum<1>(part_rays, rays_prefix, s, a);
    slice_sum<1>(part_pix, pix_prefix, s, b);
    if (threadIdx.x == 0) {
        sc[s].objective = a[0] + b[0];
        sc[s].objective_iter = sc[s].iteration;
    }
}

// ---- state set-up -------------------------------------------------------------------------------

// x_c = max(0, x_c), x_p = kappa x_c, for slices without a given start; slices with one copy x0
__global__ void __launch_bounds__(256) k_init_image(const SliceDesc* __restrict__ dsl, BlockMap pix,
                                                    const int* __restrict__ has_x0, const float2* __restrict__ x0,
                                                    float2* __restrict__ x, float kappa) {
    int local;
    const int s = slice_of(pix, blockIdx.x, local);
    const SliceDesc& d = dsl[s];
    const int64_t k = (int64_t)local * 256 + threadIdx.x;
    if (k >= (int64_t)d.g.nx * d.g.ny) return;
    const int64_t e = d.img_off + k;
    if (has_x0[s]) {
        x[e] = __ldg(x0 + e);
    } else {
        const float c = fmaxf(0.f, x[e].x);
        x[e] = make_float2(c, kappa * c);
    }
}

// y = D x, u^y = 0, z = x, u^z = 0 (image blocks); a = R x, u^a = 0, mu = mu0 (ray blocks)
template <class S2>
__global__ void __launch_bounds__(256) k_state_from_image(const SliceDesc* __restrict__ dsl, BlockMap pix, int nblk_pix,
                                                          BlockMap rays, const float2* __restrict__ x,
                                                          float4* __restrict__ y, float4* __restrict__ uy,
                                                          float2* __restrict__ z, float2* __restrict__ uz,
                                                          const S2* __restrict__ Rx, S2* __restrict__ a,
                                                          S2* __restrict__ ua, float* __restrict__ mu, float mu0) {
    int local;
    if ((int)blockIdx.x < nblk_pix) {
        const int s = slice_of(pix, blockIdx.x, local);
        const SliceDesc& d = dsl[s];
        const int nx = d.g.nx, ny = d.g.ny;
        const int64_t k = (int64_t)local * 256 + threadIdx.x;
        if (k >= (int64_t)nx * ny) return;
        const int j = (int)(k / nx), i = (int)(k % nx);
        const float2* xs = x + d.img_off;
        const float2 xc = __ldg(xs + k);
        float4 g = make_float4(0.f, 0.f, 0.f, 0.f);
        if (i < nx - 1) {
            const float2 rr = __ldg(xs + k + 1);
            g.x = rr.x - xc.x;
            g.z = rr.y - xc.y;
        }
        if (j < ny - 1) {
            const float2 uu = __ldg(xs + k + nx);
            g.y = uu.x - xc.x;
            g.w = uu.y - xc.y;
        }
        const int64_t e = d.img_off + k;
        y[e] = g;
        uy[e] = make_float4(0.f, 0.f, 0.f, 0.f);
        z[e] = xc;
        uz[e] = make_float2(0.f, 0.f);
    } else {
        const int s = slice_of(rays, blockIdx.x - nblk_pix, local);
        const SliceDesc& d = dsl[s];
        const int64_t k = (int64_t)local * 256 + threadIdx.x;
        if (k >= (int64_t)d.g.nv * d.g.nb) return;
        const int64_t e = d.sino_off + k;
        a[e] = Rx[e];
        st2(ua + e, make_float2(0.f, 0.f));
        mu[e] = mu0;
    }
}

__global__ void k_reset_scalars(SliceScalars* __restrict__ sc, int B, double rho_c, double rho_p) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= B) return;
    SliceScalars v = {};
    v.rho[0] = rho_c;
    v.rho[1] = rho_p;
    v.factor[0] = v.factor[1] = 1.0;
    v.rho_f[0] = (float)rho_c;
    v.rho_f[1] = (float)rho_p;
    v.ifactor_f[0] = v.ifactor_f[1] = 1.0f;
    v.xi_num[0] = v.xi_num[1] = nan("");
    v.xi_den[0] = v.xi_den[1] = nan("");
    v.objective = nan("");
    v.objective_iter = -1;
    sc[s] = v;
}

// measurements: four planar float arrays (staged) -> float4 per ray of slice s
__global__ void k_pack_meas(const float* __restrict__ st, int64_t n, float4* __restrict__ meas) {
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    meas[r] = make_float4(st[r], st[n + r], st[2 * n + r], st[3 * n + r]);
}

// planar [2][n] -> interleaved float2
__global__ void k_interleave(const float* __restrict__ in, int64_t n, float2* __restrict__ out) {
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    out[r] = make_float2(in[r], in[n + r]);
}

// interleaved {c, p} [n] -> planar float [2][n]
template <class S2>
__global__ void k_deinterleave2(const S2* __restrict__ in, int64_t n, float* __restrict__ out) {
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    const float2 v = ld2(in + r);
    out[r] = v.x;
    out[n + r] = v.y;
}

// float4 {xc, yc, xp, yp} [n] -> planar [2 basis][2 component][n]
__global__ void k_deinterleave4(const float4* __restrict__ in, int64_t n, float* __restrict__ out) {
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    const float4 v = in[r];
    out[r] = v.x;
    out[n + r] = v.y;
    out[2 * n + r] = v.z;
    out[3 * n + r] = v.w;
}

// plain CG (no preconditioner): s = r and <r, r> per row block, in the preconditioner's slot layout
__global__ void __launch_bounds__(256) k_identity_precond(const SliceDesc* __restrict__ dsl, BlockMap rows,
                                                          const float2* __restrict__ r, float2* __restrict__ s,
                                                          double* __restrict__ partial) {
    int j;
    const int sl = slice_of(rows, blockIdx.x, j);
    const SliceDesc& d = dsl[sl];
    const size_t row = d.img_off + (size_t)j * d.g.nx;
    double acc[2] = {0.0, 0.0};
    for (int t = threadIdx.x; t < d.g.nx; t += blockDim.x) {
        const float2 v = __ldg(r + row + t);
        s[row + t] = v;
        acc[0] += (double)v.x * v.x;
        acc[1] += (double)v.y * v.y;
    }
    block_partials<2>(acc, partial);
}

// ---- launchers -----------------------------------------------------------------------------------

void launch_identity_precond(const SliceDesc* d, const BlockMap& rows, int nrows, const float2* r, float2* s,
                             double* partial, cudaStream_t st) {
    k_identity_precond<<<nrows, 256, 0, st>>>(d, rows, r, s, partial);
}

static unsigned nb(int64_t n, int t = 256) { return (unsigned)((n + t - 1) / t); }

#define DISPATCH_S2(prec, call)                                                  \
    do {                                                                          \
        if ((prec) == PREC_F16) {                                                 \
            using S2 = __half2;                                                   \
            call;                                                                 \
        } else if ((prec) == PREC_BF16) {                                         \
            using S2 = __nv_bfloat162;                                            \
            call;                                                                 \
        } else {                                                                  \
            using S2 = float2;                                                    \
            call;                                                                 \
        }                                                                         \
    } while (0)

void launch_sino_resid(const SliceDesc* d, const BlockMap& rays, int nr, const void* a, const void* ua,
                       const void* Rx, void* b, int prec, cudaStream_t st) {
    DISPATCH_S2(prec, (k_sino_resid<S2><<<nr, 256, 0, st>>>(d, rays, (const S2*)a, (const S2*)ua, (const S2*)Rx,
                                                            (S2*)b)));
}
void launch_rs_reduce(const double* part, const int* rows_prefix, SliceScalars* sc, int B, int first, cudaStream_t st) {
    k_rs_reduce<<<B, 256, 0, st>>>(part, rows_prefix, sc, first);
}
void launch_alpha(const double* part, const int* bp_prefix, SliceScalars* sc, int B, cudaStream_t st) {
    k_alpha<<<B, 256, 0, st>>>(part, bp_prefix, sc);
}
void launch_cg_update(const SliceDesc* d, const BlockMap& pix, int np, const BlockMap& rays, int nr,
                      const SliceScalars* sc, float2* x, const float2* p, float2* r, const float2* Ap, void* Rx,
                      const void* q, int last, int prec, cudaStream_t st) {
    DISPATCH_S2(prec, (k_cg_update<S2><<<np + nr, 256, 0, st>>>(d, pix, np, rays, sc, x, p, r, Ap, (S2*)Rx,
                                                                 (const S2*)q, last)));
}
void launch_cg_p(const SliceDesc* d, const BlockMap& pix, int np, const SliceScalars* sc, const float2* s, float2* p,
                 cudaStream_t st) {
    k_cg_p<<<np, 256, 0, st>>>(d, pix, sc, s, p);
}
void launch_image_update(const SliceDesc* d, const BlockMap& pix, int np, const SliceScalars* sc, double lam_c,
                         double lam_p, const float2* x, float4* y, float4* uy, float2* z, float2* uz, double* partial,
                         cudaStream_t st) {
    k_image_update<<<np, 256, 0, st>>>(d, pix, sc, lam_c, lam_p, x, y, uy, z, uz, partial);
}
void launch_rho_update(const double* part_udm, const int* rays_prefix, const double* part_img, const int* pix_prefix,
                       SliceScalars* sc, int B, double mu_b, double tau, cudaStream_t st) {
    k_rho_update<<<B, 256, 0, st>>>(part_udm, rays_prefix, part_img, pix_prefix, sc, mu_b, tau);
}
void launch_dual_rescale(const SliceDesc* d, int B, const SliceScalars* sc, float4* uy, float2* uz, void* ua, int prec,
                         cudaStream_t st) {
    // about eight blocks per SM over the batch, at least one per slice
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int G = std::max(1, std::min(1024, (8 * std::max(sms, 1) + B - 1) / B));
    DISPATCH_S2(prec, (k_dual_rescale<S2><<<B * G, 256, 0, st>>>(d, G, sc, uy, uz, (S2*)ua)));
}
void launch_xi(const SliceDesc* d, const BlockMap& pix, int np, const float2* x, const float2* truth, double* partial,
               SliceScalars* sc, int B, cudaStream_t st) {
    k_xi_partials<<<np, 256, 0, st>>>(d, pix, x, truth, partial);
    k_xi_reduce<<<B, 256, 0, st>>>(partial, pix.prefix, sc);
}
void launch_objective_tv(const SliceDesc* d, const BlockMap& pix, int np, const float2* x, double lam_c, double lam_p,
                         double* partial, cudaStream_t st) {
    k_objective_tv<<<np, 256, 0, st>>>(d, pix, x, lam_c, lam_p, partial);
}
void launch_objective_reduce(const double* part_rays, const int* rays_prefix, const double* part_pix,
                             const int* pix_prefix, SliceScalars* sc, int B, cudaStream_t st) {
    k_objective_reduce<<<B, 256, 0, st>>>(part_rays, rays_prefix, part_pix, pix_prefix, sc);
}
void launch_xi_reduce(const double* partial, const int* pix_prefix, SliceScalars* sc, int B, cudaStream_t st) {
    k_xi_reduce<<<B, 256, 0, st>>>(partial, pix_prefix, sc);
}
void launch_init_image(const SliceDesc* d, const BlockMap& pix, int np, const int* has_x0, const float2* x0,
                       float2* x, float kappa, cudaStream_t st) {
    k_init_image<<<np, 256, 0, st>>>(d, pix, has_x0, x0, x, kappa);
}
void launch_state_from_image(const SliceDesc* d, const BlockMap& pix, int np, const BlockMap& rays, int nr,
                             const float2* x, float4* y, float4* uy, float2* z, float2* uz, const void* Rx,
                             void* a, void* ua, float* mu, float mu0, int prec, cudaStream_t st) {
    DISPATCH_S2(prec, (k_state_from_image<S2><<<np + nr, 256, 0, st>>>(d, pix, np, rays, x, y, uy, z, uz,
                                                                        (const S2*)Rx, (S2*)a, (S2*)ua, mu, mu0)));
}
void launch_reset_scalars(SliceScalars* sc, int B, double rho_c, double rho_p, cudaStream_t st) {
    k_reset_scalars<<<nb(B, 64), 64, 0, st>>>(sc, B, rho_c, rho_p);
}
void launch_pack_meas(const float* staged, int64_t n, float4* meas, cudaStream_t st) {
    k_pack_meas<<<nb(n), 256, 0, st>>>(staged, n, meas);
}
void launch_interleave(const float* in, int64_t n, float2* out, cudaStream_t st) {
    k_interleave<<<nb(n), 256, 0, st>>>(in, n, out);
}
void launch_deinterleave2(const void* in, int64_t n, float* out, int prec, cudaStream_t st) {
    DISPATCH_S2(prec, (k_deinterleave2<S2><<<nb(n), 256, 0, st>>>((const S2*)in, n, out)));
}
void launch_deinterleave4(const float4* in, int64_t n, float* out, cudaStream_t st) {
    k_deinterleave4<<<nb(n), 256, 0, st>>>(in, n, out);
}

}  // namespace dect
