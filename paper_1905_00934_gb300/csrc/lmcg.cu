// Image-side kernels of the comparison scheme LM(m) x CG(n) (Sec. 3.2: Eq. 7-8 solved by
// Levenberg-Marquardt, each LM step's linear system by n plain CG iterations; Table 1's first row).
//
// One LM step on basis b (the other basis fixed) models the data term by Gauss-Newton around the
// current projections (per ray e = sum_k w_k r_k J_k,b and g = sum_k w_k J_k,b^2, udm.cu) and adds
// the basis' augmented-Lagrangian term rho/2 ||[y; z] - C x + u||^2, C = [D; I]. The linear system
//   ((1 + mu) R^T diag(g) R + rho (D^T D + I)) d = -(R^T e - rho (D^T(y + u^y - D x) + (z + u^z - x)))
// is solved by n CG iterations from d = 0 with single-channel R / R^T (the (1 + mu) g weights are
// applied by the backprojector as it stages the rays). R d is carried through CG (R d += alpha R p),
// so the trial point needs no projection. The step is accepted iff the subproblem objective decreases:
// the change is summed per ray from the residual changes (udm.cu) and per pixel from the
// augmented-Lagrangian change, so no two large costs are subtracted. mu is per slice and basis.
// All scalars stay on the device; sums are per-block float64 partials added in a fixed order (the CG
// dot products add in float within a warp; the accept test's changes are float64 throughout).
#include <cuda_runtime.h>
#include <math.h>

#include "bp_epilogue.cuh"
#include "dect_internal.cuh"
#include "reduce.cuh"

namespace dect {

// forward differences of a single-channel image at (j, i): {along x, along y}, 0 at the last column/row
__device__ __forceinline__ float2 grad1(const float* __restrict__ a, int nx, int ny, int j, int i) {
    const float c = __ldg(a + (size_t)j * nx + i);
    float2 g = make_float2(0.f, 0.f);
    if (i < nx - 1) g.x = __ldg(a + (size_t)j * nx + i + 1) - c;
    if (j < ny - 1) g.y = __ldg(a + (size_t)(j + 1) * nx + i) - c;
    return g;
}

// (D^T D a)(j, i) for a single-channel image
__device__ __forceinline__ float dtd1(const float* __restrict__ a, int nx, int ny, int j, int i) {
    const float2 g = grad1(a, nx, ny, j, i);
    float v = 0.f;
    if (i < nx - 1) v -= g.x;
    if (i >= 1) v += grad1(a, nx, ny, j, i - 1).x;
    if (j < ny - 1) v -= g.y;
    if (j >= 1) v += grad1(a, nx, ny, j - 1, i).y;
    return v;
}

__device__ __forceinline__ float chan(float2 v, int b) { return b ? v.y : v.x; }

// scale[s] = 1 + mu_b of each slice (the damped data curvature the backprojector applies)
__global__ void k_lm_begin(const LmScalars* __restrict__ ls, float* __restrict__ scale, int B, int b) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s < B) scale[s] = (float)(1.0 + ls[s].mu[b]);
}

// Gradient of the subproblem at x from the C partial images of R^T e; r = p = -gradient, d = 0;
// partial[blk] = sum gradient^2.
__global__ void __launch_bounds__(256) k_lm_grad(const SliceDesc* __restrict__ dsl, BlockMap pix, int C,
                                                 const float* __restrict__ partial, int64_t stride, int b,
                                                 const SliceScalars* __restrict__ sc, BpEpilogue ep,
                                                 float* __restrict__ r, float* __restrict__ p,
                                                 float* __restrict__ dlt, double* __restrict__ part) {
    int local;
    const int s = slice_of(pix, blockIdx.x, local);
    const SliceDesc& d = dsl[s];
    const int nx = d.g.nx, ny = d.g.ny;
    const int64_t k = (int64_t)local * 256 + threadIdx.x;
    float acc[1] = {0.f};
    if (k < (int64_t)nx * ny) {
        const int j = (int)(k / nx), i = (int)(k % nx);
        const int64_t e = d.img_off + k;
        float rt = 0.f;
        for (int c = 0; c < C; ++c) rt += __ldg(partial + c * stride + e);
        // -(1/rho) x the augmented-Lagrangian gradient: (z + u^z - x) + D^T(y + u^y - D x), both bases
        const float4 t_ij = y_plus_u_minus_grad(ep, d.img_off, nx, ny, j, i);
        const float4 t_im = i >= 1 ? y_plus_u_minus_grad(ep, d.img_off, nx, ny, j, i - 1) : make_float4(0, 0, 0, 0);
        const float4 t_jm = j >= 1 ? y_plus_u_minus_grad(ep, d.img_off, nx, ny, j - 1, i) : make_float4(0, 0, 0, 0);
        const float2 dt = div_t(t_ij, t_im, t_jm, nx, ny, j, i);
        const float2 xc = __ldg(ep.x + e), z = __ldg(ep.z + e), uz = __ldg(ep.uz + e);
        const float epi = b ? (z.y + uz.y - xc.y + dt.y) : (z.x + uz.x - xc.x + dt.x);
        const float gr = rt - sc[s].rho_f[b] * epi;
        r[e] = -gr;
        p[e] = -gr;
        dlt[e] = 0.f;
        acc[0] = gr * gr;
    }
    block_partials<1>(acc, part);
}

// A p = (1 + mu) R^T diag(g) R p (the C partial images) + rho (D^T D p + p); partial[blk] = sum p A p
__global__ void __launch_bounds__(256) k_lm_ap(const SliceDesc* __restrict__ dsl, BlockMap pix, int C,
                                               const float* __restrict__ partial, int64_t stride, int b,
                                               const SliceScalars* __restrict__ sc, const float* __restrict__ p,
                                               float* __restrict__ Ap, double* __restrict__ part) {
    int local;
    const int s = slice_of(pix, blockIdx.x, local);
    const SliceDesc& d = dsl[s];
    const int nx = d.g.nx, ny = d.g.ny;
    const int64_t k = (int64_t)local * 256 + threadIdx.x;
    float acc[1] = {0.f};
    if (k < (int64_t)nx * ny) {
        const int j = (int)(k / nx), i = (int)(k % nx);
        const int64_t e = d.img_off + k;
        float rt = 0.f;
        for (int c = 0; c < C; ++c) rt += __ldg(partial + c * stride + e);
        const float* ps = p + d.img_off;
        const float pv = __ldg(ps + k);
        const float a = rt + sc[s].rho_f[b] * (dtd1(ps, nx, ny, j, i) + pv);
        Ap[e] = a;
        acc[0] = pv * a;
    }
    block_partials<1>(acc, part);
}

// alpha = rr / <p, A p> per slice
__global__ void __launch_bounds__(256) k_lm_alpha(const double* __restrict__ part, const int* __restrict__ prefix,
                                                  LmScalars* __restrict__ ls) {
    const int s = blockIdx.x;
    double v[1];
    slice_sum<1>(part, prefix, s, v);
    if (threadIdx.x == 0) ls[s].alpha = v[0] > 0.0 ? ls[s].rr / v[0] : 0.0;
}

// rr = <r, r>; after the first CG step also beta = rr_new / rr
__global__ void __launch_bounds__(256) k_lm_rr(const double* __restrict__ part, const int* __restrict__ prefix,
                                               LmScalars* __restrict__ ls, int first) {
    const int s = blockIdx.x;
    double v[1];
    slice_sum<1>(part, prefix, s, v);
    if (threadIdx.x == 0) {
        if (!first) ls[s].beta = ls[s].rr > 0.0 ? v[0] / ls[s].rr : 0.0;
        ls[s].rr = v[0];
    }
}

// d += alpha p and (unless last) r -= alpha A p over the image blocks, with partial sums of r^2;
// R d += alpha R p over the ray blocks
__global__ void __launch_bounds__(256) k_lm_cg(const SliceDesc* __restrict__ dsl, BlockMap pix, int nblk_pix,
                                               BlockMap rays, const LmScalars* __restrict__ ls,
                                               float* __restrict__ dlt, const float* __restrict__ p,
                                               float* __restrict__ r, const float* __restrict__ Ap,
                                               float* __restrict__ Rd, const float* __restrict__ q, int last,
                                               double* __restrict__ part) {
    int local;
    const bool img = (int)blockIdx.x < nblk_pix;
    const int s = img ? slice_of(pix, blockIdx.x, local) : slice_of(rays, blockIdx.x - nblk_pix, local);
    const SliceDesc& d = dsl[s];
    const float alpha = (float)ls[s].alpha;
    const int64_t k = (int64_t)local * 256 + threadIdx.x;
    if (img) {
        float acc[1] = {0.f};
        if (k < (int64_t)d.g.nx * d.g.ny) {
            const int64_t e = d.img_off + k;
            const float pv = p[e], dv = dlt[e];
            const float av = last ? 0.f : Ap[e], rv = last ? 0.f : r[e];  // loads before stores
            dlt[e] = fmaf(alpha, pv, dv);
            if (!last) {
                const float rn = fmaf(-alpha, av, rv);
                r[e] = rn;
                acc[0] = rn * rn;
            }
        }
        block_partials<1>(acc, part);
    } else if (k < (int64_t)d.g.nv * d.g.nb) {
        const int64_t e = d.sino_off + k;
        Rd[e] = fmaf(alpha, q[e], Rd[e]);
    }
}

// p = r + beta p
__global__ void __launch_bounds__(256) k_lm_p(const SliceDesc* __restrict__ dsl, BlockMap pix,
                                              const LmScalars* __restrict__ ls, const float* __restrict__ r,
                                              float* __restrict__ p) {
    int local;
    const int s = slice_of(pix, blockIdx.x, local);
    const SliceDesc& d = dsl[s];
    const int64_t k = (int64_t)local * 256 + threadIdx.x;
    if (k >= (int64_t)d.g.nx * d.g.ny) return;
    const int64_t e = d.img_off + k;
    p[e] = fmaf((float)ls[s].beta, p[e], r[e]);
}

// Change of the augmented-Lagrangian term of basis b for x -> x + d, per pixel (its rows of C):
// 1/2 rho (|D d|^2 - 2 <D d, y + u^y - D x> + d^2 - 2 d (z + u^z - x)); partial[blk] = sum.
__global__ void __launch_bounds__(256) k_lm_al_delta(const SliceDesc* __restrict__ dsl, BlockMap pix, int b,
                                                     const SliceScalars* __restrict__ sc, BpEpilogue ep,
                                                     const float* __restrict__ dlt, double* __restrict__ part) {
    int local;
    const int s = slice_of(pix, blockIdx.x, local);
    const SliceDesc& d = dsl[s];
    const int nx = d.g.nx, ny = d.g.ny;
    const int64_t k = (int64_t)local * 256 + threadIdx.x;
    double acc[1] = {0.0};
    if (k < (int64_t)nx * ny) {
        const int j = (int)(k / nx), i = (int)(k % nx);
        const int64_t e = d.img_off + k;
        const float4 t4 = y_plus_u_minus_grad(ep, d.img_off, nx, ny, j, i);
        const float tx = b ? t4.z : t4.x, ty = b ? t4.w : t4.y;
        const float2 gd = grad1(dlt + d.img_off, nx, ny, j, i);
        const float dv = __ldg(dlt + e);
        const float2 xc = __ldg(ep.x + e), z = __ldg(ep.z + e), uz = __ldg(ep.uz + e);
        const float sv = chan(z, b) + chan(uz, b) - chan(xc, b);
        const double v = (double)gd.x * gd.x + (double)gd.y * gd.y - 2.0 * ((double)gd.x * tx + (double)gd.y * ty) +
                         (double)dv * dv - 2.0 * (double)dv * sv;
        acc[0] = 0.5 * sc[s].rho[b] * v;
    }
    block_partials<1>(acc, part);
}

// accept iff the subproblem objective decreased; mu / 10 or * 10 (clamped); scale = 1 + mu
__global__ void __launch_bounds__(256) k_lm_decide(const double* __restrict__ part_ray,
                                                   const int* __restrict__ rays_prefix,
                                                   const double* __restrict__ part_pix,
                                                   const int* __restrict__ pix_prefix, LmScalars* __restrict__ ls,
                                                   float* __restrict__ scale, int b) {
    const int s = blockIdx.x;
    double a[1], c[1];
    slice_sum<1>(part_ray, rays_prefix, s, a);
    slice_sum<1>(part_pix, pix_prefix, s, c);
    if (threadIdx.x == 0) {
        const double dcost = a[0] + c[0];
        const bool acc = isfinite(dcost) && dcost < 0.0;
        double mu = ls[s].mu[b] * (acc ? 0.1 : 10.0);
        mu = fmin(fmax(mu, 1e-10), 1e10);
        ls[s].mu[b] = mu;
        ls[s].dcost = dcost;
        ls[s].accept = acc ? 1 : 0;
        scale[s] = (float)(1.0 + mu);
    }
}

// accepted slices: x_b += d over the image blocks, (R x)_b += R d over the ray blocks
__global__ void __launch_bounds__(256) k_lm_accept(const SliceDesc* __restrict__ dsl, BlockMap pix, int nblk_pix,
                                                   BlockMap rays, const LmScalars* __restrict__ ls, int b,
                                                   float2* __restrict__ x, const float* __restrict__ dlt,
                                                   float2* __restrict__ Rx, const float* __restrict__ Rd) {
    int local;
    const bool img = (int)blockIdx.x < nblk_pix;
    const int s = img ? slice_of(pix, blockIdx.x, local) : slice_of(rays, blockIdx.x - nblk_pix, local);
    if (!ls[s].accept) return;
    const SliceDesc& d = dsl[s];
    const int64_t k = (int64_t)local * 256 + threadIdx.x;
    if (img) {
        if (k >= (int64_t)d.g.nx * d.g.ny) return;
        const int64_t e = d.img_off + k;
        float2 v = x[e];
        if (b) v.y += dlt[e]; else v.x += dlt[e];
        x[e] = v;
    } else {
        if (k >= (int64_t)d.g.nv * d.g.nb) return;
        const int64_t e = d.sino_off + k;
        float2 v = Rx[e];
        if (b) v.y += Rd[e]; else v.x += Rd[e];
        Rx[e] = v;
    }
}

__global__ void k_lm_reset(LmScalars* __restrict__ ls, int B, double mu0) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= B) return;
    LmScalars v{};
    v.mu[0] = v.mu[1] = mu0;
    ls[s] = v;
}

// ---- launchers ------------------------------------------------------------------------------------

void launch_lm_reset(LmScalars* ls, int B, double mu0, cudaStream_t st) {
    k_lm_reset<<<(B + 127) / 128, 128, 0, st>>>(ls, B, mu0);
}
void launch_lm_begin(const LmScalars* ls, float* scale, int B, int b, cudaStream_t st) {
    k_lm_begin<<<(B + 127) / 128, 128, 0, st>>>(ls, scale, B, b);
}
void launch_lm_grad(const SliceDesc* dsl, const BlockMap& pix, int npix, int C, const float* partial, int64_t stride,
                    int b, const SliceScalars* sc, const BpEpilogue& ep, float* r, float* p, float* dlt, double* part,
                    cudaStream_t st) {
    k_lm_grad<<<npix, 256, 0, st>>>(dsl, pix, C, partial, stride, b, sc, ep, r, p, dlt, part);
}
void launch_lm_ap(const SliceDesc* dsl, const BlockMap& pix, int npix, int C, const float* partial, int64_t stride,
                  int b, const SliceScalars* sc, const float* p, float* Ap, double* part, cudaStream_t st) {
    k_lm_ap<<<npix, 256, 0, st>>>(dsl, pix, C, partial, stride, b, sc, p, Ap, part);
}
void launch_lm_alpha(const double* part, const int* prefix, LmScalars* ls, int B, cudaStream_t st) {
    k_lm_alpha<<<B, 256, 0, st>>>(part, prefix, ls);
}
void launch_lm_rr(const double* part, const int* prefix, LmScalars* ls, int B, int first, cudaStream_t st) {
    k_lm_rr<<<B, 256, 0, st>>>(part, prefix, ls, first);
}
void launch_lm_cg(const SliceDesc* dsl, const BlockMap& pix, int npix, const BlockMap& rays, int nray,
                  const LmScalars* ls, float* dlt, const float* p, float* r, const float* Ap, float* Rd, const float* q,
                  int last, double* part, cudaStream_t st) {
    k_lm_cg<<<npix + nray, 256, 0, st>>>(dsl, pix, npix, rays, ls, dlt, p, r, Ap, Rd, q, last, part);
}
void launch_lm_p(const SliceDesc* dsl, const BlockMap& pix, int npix, const LmScalars* ls, const float* r, float* p,
                 cudaStream_t st) {
    k_lm_p<<<npix, 256, 0, st>>>(dsl, pix, ls, r, p);
}
void launch_lm_al_delta(const SliceDesc* dsl, const BlockMap& pix, int npix, int b, const SliceScalars* sc,
                        const BpEpilogue& ep, const float* dlt, double* part, cudaStream_t st) {
    k_lm_al_delta<<<npix, 256, 0, st>>>(dsl, pix, b, sc, ep, dlt, part);
}
void launch_lm_decide(const double* part_ray, const int* rays_prefix, const double* part_pix, const int* pix_prefix,
                      LmScalars* ls, float* scale, int B, int b, cudaStream_t st) {
    k_lm_decide<<<B, 256, 0, st>>>(part_ray, rays_prefix, part_pix, pix_prefix, ls, scale, b);
}
void launch_lm_accept(const SliceDesc* dsl, const BlockMap& pix, int npix, const BlockMap& rays, int nray,
                      const LmScalars* ls, int b, float2* x, const float* dlt, float2* Rx, const float* Rd,
                      cudaStream_t st) {
    k_lm_accept<<<npix + nray, 256, 0, st>>>(dsl, pix, npix, rays, ls, b, x, dlt, Rx, Rd);
}

}  // namespace dect
