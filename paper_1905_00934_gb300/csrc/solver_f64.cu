// Float64 path of the ADMM solver (storage = DECT_STORE_F64): one UDM(m)-PCG(n) iteration
// (Sec. 3.3) with every vector, scalar and operation in float64, for workloads whose photoelectric
// signal lies below float32 resolution (the PE basis decays as E^-3, Sec. 1, so with a 1 keV
// reference its share of the attenuation is ~1e-7).
//
// Layout (per slice, stacked like the float32 path, planar per basis):
//   images     [2][ny][nx] at 2 * img_off (Compton plane, then PE plane)
//   y, u^y     [2 basis][2 component][ny][nx] at 4 * img_off
//   sinograms  [2][V][Nb] at 2 * sino_off; LM damping mu [V][Nb] at sino_off
//   FFT grid   double2 [py][px] at fft_off; H, H without D [py][px] at h_off
// The element-wise kernels run over the batch's pixel / ray block maps (256 per block, as in the
// float32 path), so their partial sums land in the same slots and the same reduction kernels
// (CG alpha / beta, residual balancing, xi) finish them. The projector pair is the float64
// thread-per-ray / thread-per-pixel gather of projector_f64.cu, launched per slice. Arithmetic follows
// the oracle's operation order where it is written out (Eq. 9-13); the preconditioner transforms
// Compton + i PE in one complex FFT (H is real and even, so the two parts stay separate).
#include <cuda_runtime.h>
#include <math.h>

#include "dect_internal.cuh"
#include "reduce.cuh"

namespace dect {

__device__ __forceinline__ int64_t np_of(const SliceDesc& d) { return (int64_t)d.g.nx * d.g.ny; }
__device__ __forceinline__ int64_t nr_of(const SliceDesc& d) { return (int64_t)d.g.nv * d.g.nb; }

// ---- Eq. 12 pieces -------------------------------------------------------------------------------

// b = a + u^a - R x
__global__ void __launch_bounds__(256) k64_sino_resid(const SliceDesc* __restrict__ dsl, BlockMap rays,
                                                      const double* __restrict__ a, const double* __restrict__ ua,
                                                      const double* __restrict__ Rx, double* __restrict__ b) {
    int local;
    const SliceDesc& d = dsl[slice_of(rays, blockIdx.x, local)];
    const int64_t nr = nr_of(d), k = (int64_t)local * 256 + threadIdx.x;
    if (k >= nr) return;
    for (int c = 0; c < 2; ++c) {
        const int64_t e = 2 * d.sino_off + c * nr + k;
        b[e] = a[e] + ua[e] - Rx[e];
    }
}

__device__ __forceinline__ double at64(const double* __restrict__ im, int nx, int ny, int j, int i) {
    return (i < 0 || i >= nx || j < 0 || j >= ny) ? 0.0 : im[(size_t)j * nx + i];
}

// forward differences {along x, along y} at (j, i), zero at the last column / row
__device__ __forceinline__ double2 grad64(const double* __restrict__ x, int nx, int ny, int j, int i) {
    const double c = x[(size_t)j * nx + i];
    return make_double2(i < nx - 1 ? x[(size_t)j * nx + i + 1] - c : 0.0, j < ny - 1 ? x[(size_t)(j + 1) * nx + i] - c : 0.0);
}

// (D^T t)(j, i) from t at (j, i), (j, i-1), (j-1, i), accumulated in the order of the adjoint's
// four terms: -t_x(j, i), +t_x(j, i-1), -t_y(j, i), +t_y(j-1, i)
__device__ __forceinline__ double div64(double2 t_ij, double2 t_im, double2 t_jm, int nx, int ny, int j, int i) {
    double o = 0.0;
    if (i < nx - 1) o -= t_ij.x;
    if (i >= 1) o += t_im.x;
    if (j < ny - 1) o -= t_ij.y;
    if (j >= 1) o += t_jm.y;
    return o;
}

// t = y + u^y - D x at (j, i) for one basis (y, u^y planes of that basis: x-component, then y-component)
__device__ __forceinline__ double2 yu_minus_grad(const double* __restrict__ y, const double* __restrict__ uy,
                                                 const double* __restrict__ x, int nx, int ny, int64_t np, int j,
                                                 int i) {
    const size_t e = (size_t)j * nx + i;
    const double2 g = grad64(x, nx, ny, j, i);
    return make_double2(y[e] + uy[e] - g.x, y[np + e] + uy[np + e] - g.y);
}

// r0 = R^T b + (z + u^z - x) [+ D^T(y + u^y - D x)]; RTb holds R^T b (planar per slice)
__global__ void __launch_bounds__(256) k64_r0(const SliceDesc* __restrict__ dsl, BlockMap pix,
                                              const double* __restrict__ RTb, const double* __restrict__ x,
                                              const double* __restrict__ y, const double* __restrict__ uy,
                                              const double* __restrict__ z, const double* __restrict__ uz,
                                              double* __restrict__ r, int with_grad) {
    int local;
    const SliceDesc& d = dsl[slice_of(pix, blockIdx.x, local)];
    const int nx = d.g.nx, ny = d.g.ny;
    const int64_t np = np_of(d), k = (int64_t)local * 256 + threadIdx.x;
    if (k >= np) return;
    const int j = (int)(k / nx), i = (int)(k % nx);
    for (int c = 0; c < 2; ++c) {
        const int64_t base = 2 * d.img_off + c * np, e = base + k;
        double v = RTb[e] + (z[e] + uz[e] - x[e]);
        if (with_grad) {
            const double* xs = x + base;
            const double* ys = y + 4 * d.img_off + 2 * c * np;
            const double* us = uy + 4 * d.img_off + 2 * c * np;
            const double2 tij = yu_minus_grad(ys, us, xs, nx, ny, np, j, i);
            const double2 tim = i >= 1 ? yu_minus_grad(ys, us, xs, nx, ny, np, j, i - 1) : make_double2(0.0, 0.0);
            const double2 tjm = j >= 1 ? yu_minus_grad(ys, us, xs, nx, ny, np, j - 1, i) : make_double2(0.0, 0.0);
            v += div64(tij, tim, tjm, nx, ny, j, i);
        }
        r[e] = v;
    }
}

// A p = R^T q + p [+ D^T D p]; partial[2 blk + c] = <p_c, (A p)_c>
__global__ void __launch_bounds__(256) k64_ap(const SliceDesc* __restrict__ dsl, BlockMap pix,
                                              const double* __restrict__ RTq, const double* __restrict__ p,
                                              double* __restrict__ Ap, double* __restrict__ partial, int with_grad) {
    int local;
    const SliceDesc& d = dsl[slice_of(pix, blockIdx.x, local)];
    const int nx = d.g.nx, ny = d.g.ny;
    const int64_t np = np_of(d), k = (int64_t)local * 256 + threadIdx.x;
    double acc[2] = {0.0, 0.0};
    if (k < np) {
        const int j = (int)(k / nx), i = (int)(k % nx);
        for (int c = 0; c < 2; ++c) {
            const int64_t base = 2 * d.img_off + c * np, e = base + k;
            const double* ps = p + base;
            double v = RTq[e] + p[e];
            if (with_grad) {
                const double2 tij = grad64(ps, nx, ny, j, i);
                const double2 tim = i >= 1 ? grad64(ps, nx, ny, j, i - 1) : make_double2(0.0, 0.0);
                const double2 tjm = j >= 1 ? grad64(ps, nx, ny, j - 1, i) : make_double2(0.0, 0.0);
                v += div64(tij, tim, tjm, nx, ny, j, i);
            }
            Ap[e] = v;
            acc[c] = p[e] * v;
        }
    }
    block_partials<2>(acc, partial);
}

// x += alpha p, R x += alpha q, r -= alpha A p (unless last)
__global__ void __launch_bounds__(256) k64_cg_update(const SliceDesc* __restrict__ dsl, BlockMap pix, int nblk_pix,
                                                     BlockMap rays, const SliceScalars* __restrict__ sc,
                                                     double* __restrict__ x, const double* __restrict__ p,
                                                     double* __restrict__ r, const double* __restrict__ Ap,
                                                     double* __restrict__ Rx, const double* __restrict__ q, int last) {
    int local;
    const bool img = (int)blockIdx.x < nblk_pix;
    const int s = img ? slice_of(pix, blockIdx.x, local) : slice_of(rays, blockIdx.x - nblk_pix, local);
    const SliceDesc& d = dsl[s];
    const int64_t k = (int64_t)local * 256 + threadIdx.x;
    if (img) {
        const int64_t np = np_of(d);
        if (k >= np) return;
        for (int c = 0; c < 2; ++c) {
            const double al = sc[s].alpha[c];
            const int64_t e = 2 * d.img_off + c * np + k;
            x[e] = x[e] + al * p[e];
            if (!last) r[e] = r[e] - al * Ap[e];
        }
    } else {
        const int64_t nr = nr_of(d);
        if (k >= nr) return;
        for (int c = 0; c < 2; ++c) {
            const int64_t e = 2 * d.sino_off + c * nr + k;
            Rx[e] = Rx[e] + sc[s].alpha[c] * q[e];
        }
    }
}

// p = s + beta p
__global__ void __launch_bounds__(256) k64_cg_p(const SliceDesc* __restrict__ dsl, BlockMap pix,
                                                const SliceScalars* __restrict__ sc, const double* __restrict__ sv,
                                                double* __restrict__ p) {
    int local;
    const int s = slice_of(pix, blockIdx.x, local);
    const SliceDesc& d = dsl[s];
    const int64_t np = np_of(d), k = (int64_t)local * 256 + threadIdx.x;
    if (k >= np) return;
    for (int c = 0; c < 2; ++c) {
        const int64_t e = 2 * d.img_off + c * np + k;
        p[e] = sv[e] + sc[s].beta[c] * p[e];
    }
}

// ---- preconditioner: complex FFTs in float64 -----------------------------------------------------

__device__ __forceinline__ int brev64(int t, int logn) { return (int)(__brev((unsigned)t) >> (32 - logn)); }

// radix-2 decimation in time on a bit-reversed shared buffer (all threads of the block take part);
// twiddle of butterfly position pos at stage half: exp(-+ i pi pos / half)
__device__ void fft64(double2* buf, int logn, bool inverse) {
    const int n = 1 << logn;
    for (int s = 0; s < logn; ++s) {
        const int half = 1 << s;
        for (int b = threadIdx.x; b < n / 2; b += blockDim.x) {
            const int pos = b & (half - 1);
            const int i0 = ((b >> s) << (s + 1)) + pos, i1 = i0 + half;
            double sn, cs;
            sincospi((double)pos / (double)half, &sn, &cs);
            const double wi = inverse ? sn : -sn;
            const double2 u = buf[i0], v = buf[i1];
            const double tr = cs * v.x - wi * v.y, ti = cs * v.y + wi * v.x;
            buf[i0] = make_double2(u.x + tr, u.y + ti);
            buf[i1] = make_double2(u.x - tr, u.y - ti);
        }
        __syncthreads();
    }
}

// forward FFT of image row j (Compton + i PE, zero-padded to px) into Z
__global__ void __launch_bounds__(256) k64_rows_fwd(const SliceDesc* __restrict__ dsl, BlockMap rows,
                                                    const double* __restrict__ r, double2* __restrict__ Z) {
    extern __shared__ double2 zb[];
    int j;
    const SliceDesc& d = dsl[slice_of(rows, blockIdx.x, j)];
    const int nx = d.g.nx, px = d.px;
    const int64_t np = np_of(d);
    const double* rc = r + 2 * d.img_off + (size_t)j * nx;
    for (int t = threadIdx.x; t < px; t += blockDim.x)
        zb[brev64(t, d.lpx)] = t < nx ? make_double2(rc[t], rc[np + t]) : make_double2(0.0, 0.0);
    __syncthreads();
    fft64(zb, d.lpx, false);
    double2* zr = Z + d.fft_off + (size_t)j * px;
    for (int t = threadIdx.x; t < px; t += blockDim.x) zr[t] = zb[t];
}

// all py rows of a full grid (the point response)
__global__ void __launch_bounds__(256) k64_rows_full(SliceDesc d, double2* __restrict__ Z) {
    extern __shared__ double2 zb[];
    double2* zr = Z + (size_t)blockIdx.x * d.px;
    for (int t = threadIdx.x; t < d.px; t += blockDim.x) zb[brev64(t, d.lpx)] = zr[t];
    __syncthreads();
    fft64(zb, d.lpx, false);
    for (int t = threadIdx.x; t < d.px; t += blockDim.x) zr[t] = zb[t];
}

// column k: forward FFT (rows >= rows_in are zero), times H (if given), inverse FFT; rows [0, rows_out)
__global__ void __launch_bounds__(256) k64_cols(const SliceDesc* __restrict__ dsl, BlockMap cols,
                                                double2* __restrict__ Z, const double* __restrict__ H, int rows_in_all,
                                                int rows_out_all) {
    extern __shared__ double2 zb[];
    int k;
    const SliceDesc& d = dsl[slice_of(cols, blockIdx.x, k)];
    const int px = d.px, py = d.py, lp = d.lpy;
    const int rows_in = rows_in_all ? py : d.g.ny, rows_out = rows_out_all ? py : d.g.ny;
    double2* zs = Z + d.fft_off;
    for (int j = threadIdx.x; j < py; j += blockDim.x)
        zb[brev64(j, lp)] = j < rows_in ? zs[(size_t)j * px + k] : make_double2(0.0, 0.0);
    __syncthreads();
    fft64(zb, lp, false);
    if (H) {
        const double* hs = H + d.h_off;
        for (int j = threadIdx.x; j < py; j += blockDim.x) {
            const double h = hs[(size_t)j * px + k];
            zb[j] = make_double2(zb[j].x * h, zb[j].y * h);
        }
        __syncthreads();
        for (int t = threadIdx.x; t < py; t += blockDim.x) {
            const int u = brev64(t, lp);
            if (t < u) {
                const double2 a = zb[t];
                zb[t] = zb[u];
                zb[u] = a;
            }
        }
        __syncthreads();
        fft64(zb, lp, true);
    }
    for (int j = threadIdx.x; j < rows_out; j += blockDim.x) zs[(size_t)j * px + k] = zb[j];
}

// inverse FFT of row j, scaled by 1 / (px py), cropped: s = {Re, Im}; partial[2 row + c] = <r_c, s_c>
__global__ void __launch_bounds__(256) k64_rows_inv(const SliceDesc* __restrict__ dsl, BlockMap rows,
                                                    const double2* __restrict__ Z, const double* __restrict__ r,
                                                    double* __restrict__ s_out, double* __restrict__ partial) {
    extern __shared__ double2 zb[];
    int j;
    const SliceDesc& d = dsl[slice_of(rows, blockIdx.x, j)];
    const int nx = d.g.nx, px = d.px;
    const int64_t np = np_of(d);
    const double2* zr = Z + d.fft_off + (size_t)j * px;
    for (int t = threadIdx.x; t < px; t += blockDim.x) zb[brev64(t, d.lpx)] = zr[t];
    __syncthreads();
    fft64(zb, d.lpx, true);
    const double scale = 1.0 / ((double)px * (double)d.py);
    const size_t row = 2 * d.img_off + (size_t)j * nx;
    double acc[2] = {0.0, 0.0};
    for (int t = threadIdx.x; t < nx; t += blockDim.x) {
        const double sc_ = zb[t].x * scale, sp_ = zb[t].y * scale;
        s_out[row + t] = sc_;
        s_out[row + np + t] = sp_;
        acc[0] += r[row + t] * sc_;
        acc[1] += r[row + np + t] * sp_;
    }
    block_partials<2>(acc, partial);
}

// plain CG: s = r, partial[2 row + c] = <r_c, r_c>
__global__ void __launch_bounds__(256) k64_identity(const SliceDesc* __restrict__ dsl, BlockMap rows,
                                                    const double* __restrict__ r, double* __restrict__ s_out,
                                                    double* __restrict__ partial) {
    int j;
    const SliceDesc& d = dsl[slice_of(rows, blockIdx.x, j)];
    const int nx = d.g.nx;
    const int64_t np = np_of(d);
    const size_t row = 2 * d.img_off + (size_t)j * nx;
    double acc[2] = {0.0, 0.0};
    for (int t = threadIdx.x; t < nx; t += blockDim.x) {
        for (int c = 0; c < 2; ++c) {
            const double v = r[row + c * np + t];
            s_out[row + c * np + t] = v;
            acc[c] += v * v;
        }
    }
    block_partials<2>(acc, partial);
}

// point response psf (planar, first channel) wrapped onto the grid centred at index (0, 0)
__global__ void k64_embed_psf(SliceDesc d, const double* __restrict__ psf, double2* __restrict__ Z) {
    const int64_t n = (int64_t)d.px * d.py, e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    const int k = (int)(e / d.px), l = (int)(e % d.px);
    const int jc = d.g.ny / 2, ic = d.g.nx / 2;
    const int j = k < d.py / 2 ? jc + k : jc + k - d.py;
    const int i = l < d.px / 2 ? ic + l : ic + l - d.px;
    const double v = (j >= 0 && j < d.g.ny && i >= 0 && i < d.g.nx) ? psf[(size_t)j * d.g.nx + i] : 0.0;
    Z[e] = make_double2(v, 0.0);
}

// circulant model H = 1 / (max(Re P, 0) + 4 sin^2(wx/2) + 4 sin^2(wy/2) + 1), H without D; or the ramp filter
__global__ void k64_response(SliceDesc d, const double2* __restrict__ Z, double* __restrict__ H,
                             double* __restrict__ Hn, int ramp) {
    const int64_t n = (int64_t)d.px * d.py, e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    const int k = (int)(e / d.px), l = (int)(e % d.px);
    if (ramp) {
        const double K = fmax(Z[d.px / 8].x, 0.0) * (0.25 * M_PI);
        const double wy = 2.0 * M_PI * min(k, d.py - k) / d.py, wx = 2.0 * M_PI * min(l, d.px - l) / d.px;
        const double w = fmax(sqrt(wy * wy + wx * wx), 2.0 * M_PI / max(d.px, d.py));
        H[e] = Hn[e] = 1.0 / (K / w + 1.0);
        return;
    }
    const double sy = sin(0.5 * (2.0 * M_PI * k / d.py)), sx = sin(0.5 * (2.0 * M_PI * l / d.px));
    const double dhat = 4.0 * sy * sy + 4.0 * sx * sx;
    const double phat = fmax(Z[e].x, 0.0);
    H[e] = 1.0 / (phat + dhat + 1.0);
    Hn[e] = 1.0 / (phat + 1.0);
}

// ---- Eq. 13 in float64 (the oracle's Levenberg-Marquardt, step for step) -------------------------

// f_h, f_l at (ac, ap) and the Jacobian {dfh/dac, dfh/dap, dfl/dac, dfl/dap}; T = {S_h, S_l, f_KN, f_p}
__device__ __forceinline__ void fwd64(const double4_32a* __restrict__ T, int ne, double ac, double ap, double& fh,
                                      double& fl, double* J) {
    double sh = 0.0, sl = 0.0, shc = 0.0, shp = 0.0, slc = 0.0, slp = 0.0;
    for (int e = 0; e < ne; ++e) {
        const double4_32a t4 = T[e];
        const double t = exp(-t4.z * ac - t4.w * ap);
        sh += t4.x * t;
        sl += t4.y * t;
        if (J) {
            shc += t4.x * t4.z * t;
            shp += t4.x * t4.w * t;
            slc += t4.y * t4.z * t;
            slp += t4.y * t4.w * t;
        }
    }
    fh = -log(sh);
    fl = -log(sl);
    if (J) {
        J[0] = shc / sh;
        J[1] = shp / sh;
        J[2] = slc / sl;
        J[3] = slp / sl;
    }
}

struct Ray64 {
    double mh, ml, wh, wl, vc, vp, rc, rp;
};

__device__ __forceinline__ double cost64(const Ray64& q, double fh, double fl, double ac, double ap) {
    const double rh = fh - q.mh, rl = fl - q.ml;
    return 0.5 * (q.wh * rh * rh + q.wl * rl * rl) + 0.5 * (q.rc * (ac - q.vc) * (ac - q.vc) + q.rp * (ap - q.vp) * (ap - q.vp));
}

// `iters` LM iterations: Gauss-Newton system A = sum_k w_k J_k J_k^T + diag(rho), Marquardt damping
// B = A with its diagonal times (1 + mu), step -B^-1 g, kept iff the cost decreases (mu / 10, else * 10),
// mu clamped to [1e-10, 1e10]; status 0 accepted, 1 rejected, 2 non-finite or singular
__device__ void lm64(const double4_32a* __restrict__ T, int ne, const Ray64& q, int iters, double& a0, double& a1,
                     double& m, uint8_t& st) {
    for (int it = 0; it < iters; ++it) {
        double fh, fl, J[4];
        fwd64(T, ne, a0, a1, fh, fl, J);
        const double rh = fh - q.mh, rl = fl - q.ml;
        const double g0 = q.wh * rh * J[0] + q.wl * rl * J[2] + q.rc * (a0 - q.vc);
        const double g1 = q.wh * rh * J[1] + q.wl * rl * J[3] + q.rp * (a1 - q.vp);
        const double A00 = q.wh * J[0] * J[0] + q.wl * J[2] * J[2] + q.rc;
        const double A01 = q.wh * J[0] * J[1] + q.wl * J[2] * J[3];
        const double A11 = q.wh * J[1] * J[1] + q.wl * J[3] * J[3] + q.rp;
        const double B00 = A00 * (1.0 + m), B11 = A11 * (1.0 + m);
        const double det = B00 * B11 - A01 * A01;
        const double cost0 = cost64(q, fh, fl, a0, a1);
        if (!(det > 0.0) || !isfinite(det) || !isfinite(cost0)) {
            st = DECT_RAY_NONFINITE;
            break;
        }
        const double t0 = a0 + (-g0 * B11 + g1 * A01) / det;
        const double t1 = a1 + (-g1 * B00 + g0 * A01) / det;
        double fh1, fl1;
        fwd64(T, ne, t0, t1, fh1, fl1, nullptr);
        const double cost1 = cost64(q, fh1, fl1, t0, t1);
        if (!isfinite(cost1)) {
            m *= 10.0;
            st = DECT_RAY_NONFINITE;
        } else if (cost1 < cost0) {
            a0 = t0;
            a1 = t1;
            m /= 10.0;
            st = DECT_RAY_ACCEPTED;
        } else {
            m *= 10.0;
            st = DECT_RAY_REJECTED;
        }
        m = fmin(fmax(m, 1e-10), 1e10);
    }
}

__device__ __forceinline__ const double4_32a* load_tables64(const double4_32a* __restrict__ t64, int ne, double4_32a* sh) {
    for (int e = threadIdx.x; e < ne; e += blockDim.x) sh[e] = t64[e];
    __syncthreads();
    return sh;
}

// a-update (v = R x - u^a) fused with u^a += a - R x; partial[4 blk + {0,1}] = sum (a - R x)^2,
// {2,3} = sum (a - a_old)^2
__global__ void __launch_bounds__(256) k64_udm_admm(const SliceDesc* __restrict__ dsl, BlockMap rays,
                                                    const double4_32a* __restrict__ t64, int ne,
                                                    const float4* __restrict__ meas, const double* __restrict__ Rx,
                                                    double* __restrict__ ua, double* __restrict__ a,
                                                    double* __restrict__ mu, uint8_t* __restrict__ status,
                                                    const SliceScalars* __restrict__ sc, int iters,
                                                    double* __restrict__ partial) {
    extern __shared__ double4_32a tab64[];
    const double4_32a* T = load_tables64(t64, ne, tab64);
    int local;
    const int s = slice_of(rays, blockIdx.x, local);
    const SliceDesc& d = dsl[s];
    const int64_t nr = nr_of(d), k = (int64_t)local * 256 + threadIdx.x;
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    if (k < nr) {
        const int64_t ec = 2 * d.sino_off + k, ep = ec + nr, er = d.sino_off + k;
        const float4 m4 = meas[er];
        Ray64 q;
        q.mh = m4.x;
        q.ml = m4.y;
        q.wh = m4.z;
        q.wl = m4.w;
        q.vc = Rx[ec] - ua[ec];
        q.vp = Rx[ep] - ua[ep];
        q.rc = sc[s].rho[0];
        q.rp = sc[s].rho[1];
        const double oc = a[ec], op = a[ep];
        double a0 = oc, a1 = op, m = mu[er];
        uint8_t st = DECT_RAY_ACCEPTED;
        lm64(T, ne, q, iters, a0, a1, m, st);
        a[ec] = a0;
        a[ep] = a1;
        mu[er] = m;
        if (status) status[er] = st;
        ua[ec] = ua[ec] + a0 - Rx[ec];
        ua[ep] = ua[ep] + a1 - Rx[ep];
        const double rc = a0 - Rx[ec], rp = a1 - Rx[ep], dc = a0 - oc, dp = a1 - op;
        acc[0] = rc * rc;
        acc[1] = rp * rp;
        acc[2] = dc * dc;
        acc[3] = dp * dp;
    }
    block_partials<4>(acc, partial);
}

// initial decomposition: rho = (0, rho_p), v = 0, from a = (m_l / abar, 0); a = (a_c, 0), mu = mu0
__global__ void __launch_bounds__(256) k64_udm_init(const SliceDesc* __restrict__ dsl, BlockMap rays,
                                                    const double4_32a* __restrict__ t64, int ne,
                                                    const float4* __restrict__ meas, double* __restrict__ a,
                                                    double* __restrict__ mu, double rho_p, int iters, double abar,
                                                    double mu0) {
    extern __shared__ double4_32a tab64[];
    const double4_32a* T = load_tables64(t64, ne, tab64);
    int local;
    const SliceDesc& d = dsl[slice_of(rays, blockIdx.x, local)];
    const int64_t nr = nr_of(d), k = (int64_t)local * 256 + threadIdx.x;
    if (k >= nr) return;
    const float4 m4 = meas[d.sino_off + k];
    Ray64 q;
    q.mh = m4.x;
    q.ml = m4.y;
    q.wh = m4.z;
    q.wl = m4.w;
    q.vc = q.vp = 0.0;
    q.rc = 0.0;
    q.rp = rho_p;
    double a0 = (double)m4.y / abar, a1 = 0.0, m = mu0;
    uint8_t st = DECT_RAY_ACCEPTED;
    lm64(T, ne, q, iters, a0, a1, m, st);
    a[2 * d.sino_off + k] = a0;
    a[2 * d.sino_off + nr + k] = 0.0;
    mu[d.sino_off + k] = mu0;
}

// Eq. 4's data term at the projections q = R x: partial[blk] = sum 1/2 (w_h r_h^2 + w_l r_l^2)
__global__ void __launch_bounds__(256) k64_objective_rays(const SliceDesc* __restrict__ dsl, BlockMap rays,
                                                          const double4_32a* __restrict__ t64, int ne,
                                                          const float4* __restrict__ meas,
                                                          const double* __restrict__ q, double* __restrict__ partial) {
    extern __shared__ double4_32a tab64[];
    const double4_32a* T = load_tables64(t64, ne, tab64);
    int local;
    const SliceDesc& d = dsl[slice_of(rays, blockIdx.x, local)];
    const int64_t nr = nr_of(d), k = (int64_t)local * 256 + threadIdx.x;
    double acc[1] = {0.0};
    if (k < nr) {
        const float4 m4 = meas[d.sino_off + k];
        double fh, fl;
        fwd64(T, ne, q[2 * d.sino_off + k], q[2 * d.sino_off + nr + k], fh, fl, nullptr);
        const double rh = fh - m4.x, rl = fl - m4.y;
        acc[0] = 0.5 * (m4.z * rh * rh + m4.w * rl * rl);
    }
    block_partials<1>(acc, partial);
}

// Eq. 4's regulariser: partial[blk] = sum lambda_c |D x_c|_1 + lambda_p |D x_p|_1
__global__ void __launch_bounds__(256) k64_objective_tv(const SliceDesc* __restrict__ dsl, BlockMap pix,
                                                        const double* __restrict__ x, double lam_c, double lam_p,
                                                        double* __restrict__ partial) {
    int local;
    const SliceDesc& d = dsl[slice_of(pix, blockIdx.x, local)];
    const int nx = d.g.nx, ny = d.g.ny;
    const int64_t np = np_of(d), k = (int64_t)local * 256 + threadIdx.x;
    double acc[1] = {0.0};
    if (k < np) {
        const int j = (int)(k / nx), i = (int)(k % nx);
        const double2 gc = grad64(x + 2 * d.img_off, nx, ny, j, i), gp = grad64(x + 2 * d.img_off + np, nx, ny, j, i);
        acc[0] = lam_c * (fabs(gc.x) + fabs(gc.y)) + lam_p * (fabs(gp.x) + fabs(gp.y));
    }
    block_partials<1>(acc, partial);
}

// ---- Eq. 9-11 on the image side, residual sums ----------------------------------------------------

// y = shrinkage(D x - u^y, lambda / rho), z = max(0, x - u^z), u^y += y - D x, u^z += z - x;
// partial[4 blk + c] = sum (y - D x)^2 + (z - x)^2, [4 blk + 2 + c] = sum (y - y_old)^2 + (z - z_old)^2
__global__ void __launch_bounds__(256) k64_image_update(const SliceDesc* __restrict__ dsl, BlockMap pix,
                                                        const SliceScalars* __restrict__ sc, double lam_c,
                                                        double lam_p, const double* __restrict__ x,
                                                        double* __restrict__ y, double* __restrict__ uy,
                                                        double* __restrict__ z, double* __restrict__ uz,
                                                        double* __restrict__ partial) {
    int local;
    const int s = slice_of(pix, blockIdx.x, local);
    const SliceDesc& d = dsl[s];
    const int nx = d.g.nx, ny = d.g.ny;
    const int64_t np = np_of(d), k = (int64_t)local * 256 + threadIdx.x;
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    if (k < np) {
        const int j = (int)(k / nx), i = (int)(k % nx);
        for (int c = 0; c < 2; ++c) {
            const double tau = (c ? lam_p : lam_c) / sc[s].rho[c];
            const int64_t eb = 2 * d.img_off + c * np + k;
            const double2 g = grad64(x + 2 * d.img_off + c * np, nx, ny, j, i);
            const double gv[2] = {g.x, g.y};
            double pri = 0.0, dual = 0.0;
            for (int comp = 0; comp < 2; ++comp) {
                const int64_t ey = 4 * d.img_off + (2 * c + comp) * np + k;
                const double t = gv[comp] - uy[ey];
                const double mag = fabs(t) - tau;
                const double yn = mag > 0.0 ? copysign(mag, t) : 0.0;
                const double yo = y[ey];
                y[ey] = yn;
                uy[ey] = uy[ey] + yn - gv[comp];
                pri += (yn - gv[comp]) * (yn - gv[comp]);
                dual += (yn - yo) * (yn - yo);
            }
            const double zo = z[eb], zn = fmax(0.0, x[eb] - uz[eb]);
            z[eb] = zn;
            uz[eb] = uz[eb] + zn - x[eb];
            pri += (zn - x[eb]) * (zn - x[eb]);
            dual += (zn - zo) * (zn - zo);
            acc[c] = pri;
            acc[2 + c] = dual;
        }
    }
    block_partials<4>(acc, partial);
}

// scaled duals follow rho: u /= factor
__global__ void __launch_bounds__(256) k64_dual_rescale(const SliceDesc* __restrict__ dsl, BlockMap pix, int nblk_pix,
                                                        BlockMap rays, const SliceScalars* __restrict__ sc,
                                                        double* __restrict__ uy, double* __restrict__ uz,
                                                        double* __restrict__ ua) {
    int local;
    const bool img = (int)blockIdx.x < nblk_pix;
    const int s = img ? slice_of(pix, blockIdx.x, local) : slice_of(rays, blockIdx.x - nblk_pix, local);
    const double f[2] = {sc[s].factor[0], sc[s].factor[1]};
    if (f[0] == 1.0 && f[1] == 1.0) return;
    const SliceDesc& d = dsl[s];
    const int64_t k = (int64_t)local * 256 + threadIdx.x;
    if (img) {
        const int64_t np = np_of(d);
        if (k >= np) return;
        for (int c = 0; c < 2; ++c) {
            if (f[c] == 1.0) continue;
            uz[2 * d.img_off + c * np + k] /= f[c];
            for (int comp = 0; comp < 2; ++comp) uy[4 * d.img_off + (2 * c + comp) * np + k] /= f[c];
        }
    } else {
        const int64_t nr = nr_of(d);
        if (k >= nr) return;
        for (int c = 0; c < 2; ++c)
            if (f[c] != 1.0) ua[2 * d.sino_off + c * nr + k] /= f[c];
    }
}

// ---- state set-up and monitors ----------------------------------------------------------------------

// slices with a start x0 copy it (float32 planar [2][np] per slice, converted exactly); the others take
// x_c = max(0, x_c), x_p = kappa x_c
__global__ void __launch_bounds__(256) k64_init_image(const SliceDesc* __restrict__ dsl, BlockMap pix,
                                                      const int* __restrict__ has_x0, const double* __restrict__ x0,
                                                      double* __restrict__ x, double kappa) {
    int local;
    const int s = slice_of(pix, blockIdx.x, local);
    const SliceDesc& d = dsl[s];
    const int64_t np = np_of(d), k = (int64_t)local * 256 + threadIdx.x;
    if (k >= np) return;
    const int64_t ec = 2 * d.img_off + k, ep = ec + np;
    if (has_x0[s]) {
        x[ec] = x0[ec];
        x[ep] = x0[ep];
    } else {
        const double c = fmax(0.0, x[ec]);
        x[ec] = c;
        x[ep] = kappa * c;
    }
}

// y = D x, u^y = 0, z = x, u^z = 0 (pixel blocks); a = R x, u^a = 0, mu = mu0 (ray blocks)
__global__ void __launch_bounds__(256) k64_state_from_image(const SliceDesc* __restrict__ dsl, BlockMap pix,
                                                            int nblk_pix, BlockMap rays, const double* __restrict__ x,
                                                            double* __restrict__ y, double* __restrict__ uy,
                                                            double* __restrict__ z, double* __restrict__ uz,
                                                            const double* __restrict__ Rx, double* __restrict__ a,
                                                            double* __restrict__ ua, double* __restrict__ mu,
                                                            double mu0) {
    int local;
    const bool img = (int)blockIdx.x < nblk_pix;
    const SliceDesc& d = dsl[img ? slice_of(pix, blockIdx.x, local) : slice_of(rays, blockIdx.x - nblk_pix, local)];
    const int64_t k = (int64_t)local * 256 + threadIdx.x;
    if (img) {
        const int nx = d.g.nx, ny = d.g.ny;
        const int64_t np = np_of(d);
        if (k >= np) return;
        const int j = (int)(k / nx), i = (int)(k % nx);
        for (int c = 0; c < 2; ++c) {
            const int64_t e = 2 * d.img_off + c * np + k;
            const double2 g = grad64(x + 2 * d.img_off + c * np, nx, ny, j, i);
            const int64_t ey = 4 * d.img_off + 2 * c * np + k;
            y[ey] = g.x;
            y[ey + np] = g.y;
            uy[ey] = uy[ey + np] = 0.0;
            z[e] = x[e];
            uz[e] = 0.0;
        }
    } else {
        const int64_t nr = nr_of(d);
        if (k >= nr) return;
        for (int c = 0; c < 2; ++c) {
            const int64_t e = 2 * d.sino_off + c * nr + k;
            a[e] = Rx[e];
            ua[e] = 0.0;
        }
        mu[d.sino_off + k] = mu0;
    }
}

// partial[4 blk + {0,1}] = sum (x - x*)^2 per basis, {2,3} = sum x*^2 (truth: float2 {c, p})
__global__ void __launch_bounds__(256) k64_xi_partials(const SliceDesc* __restrict__ dsl, BlockMap pix,
                                                       const double* __restrict__ x, const float2* __restrict__ truth,
                                                       double* __restrict__ partial) {
    int local;
    const SliceDesc& d = dsl[slice_of(pix, blockIdx.x, local)];
    const int64_t np = np_of(d), k = (int64_t)local * 256 + threadIdx.x;
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    if (k < np) {
        const float2 t = truth[d.img_off + k];
        const double dc = x[2 * d.img_off + k] - t.x, dp = x[2 * d.img_off + np + k] - t.y;
        acc[0] = dc * dc;
        acc[1] = dp * dp;
        acc[2] = (double)t.x * t.x;
        acc[3] = (double)t.y * t.y;
    }
    block_partials<4>(acc, partial);
}

// float32 planar [2][n] (per slice, n elements at offset `off`) -> float64 planar at 2 * off
__global__ void k64_from_f32(const float* __restrict__ in, int64_t n, double* __restrict__ out) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e < 2 * n) out[e] = (double)in[e];
}

// ---- launchers --------------------------------------------------------------------------------------

static unsigned nblocks(int64_t n, int t = 256) { return (unsigned)((n + t - 1) / t); }

void launch64_sino_resid(const SliceDesc* d, const BlockMap& rays, int nr, const double* a, const double* ua,
                         const double* Rx, double* b, cudaStream_t st) {
    k64_sino_resid<<<nr, 256, 0, st>>>(d, rays, a, ua, Rx, b);
}
void launch64_r0(const SliceDesc* d, const BlockMap& pix, int np, const double* RTb, const F64Vecs& v, double* r,
                 bool with_grad, cudaStream_t st) {
    k64_r0<<<np, 256, 0, st>>>(d, pix, RTb, v.x, v.y, v.uy, v.z, v.uz, r, with_grad ? 1 : 0);
}
void launch64_ap(const SliceDesc* d, const BlockMap& pix, int np, const double* RTq, const double* p, double* Ap,
                 double* partial, bool with_grad, cudaStream_t st) {
    k64_ap<<<np, 256, 0, st>>>(d, pix, RTq, p, Ap, partial, with_grad ? 1 : 0);
}
void launch64_cg_update(const SliceDesc* d, const BlockMap& pix, int np, const BlockMap& rays, int nr,
                        const SliceScalars* sc, const F64Vecs& v, int last, cudaStream_t st) {
    k64_cg_update<<<np + nr, 256, 0, st>>>(d, pix, np, rays, sc, v.x, v.p, v.r, v.Ap, v.Rx, v.q, last);
}
void launch64_cg_p(const SliceDesc* d, const BlockMap& pix, int np, const SliceScalars* sc, const double* s, double* p,
                   cudaStream_t st) {
    k64_cg_p<<<np, 256, 0, st>>>(d, pix, sc, s, p);
}
void launch64_precond(const SliceDesc* d, const BlockMap& rows, int nrows, const BlockMap& cols, int ncols,
                      const double* H, const double* r, double* s, double2* Z, double* partial, int max_px, int max_py,
                      cudaStream_t st) {
    if (!H) {
        k64_identity<<<nrows, 256, 0, st>>>(d, rows, r, s, partial);
        return;
    }
    k64_rows_fwd<<<nrows, 256, sizeof(double2) * max_px, st>>>(d, rows, r, Z);
    k64_cols<<<ncols, 256, sizeof(double2) * max_py, st>>>(d, cols, Z, H, 0, 0);
    k64_rows_inv<<<nrows, 256, sizeof(double2) * max_px, st>>>(d, rows, Z, r, s, partial);
}
void launch64_response(const SliceDesc* d_dev, const SliceDesc& d, const BlockMap& cols, int ncols, const double* psf,
                       double2* Z, double* H, double* Hn, bool ramp, cudaStream_t st) {
    const int64_t n = (int64_t)d.px * d.py;
    k64_embed_psf<<<nblocks(n), 256, 0, st>>>(d, psf, Z);
    k64_rows_full<<<d.py, 256, sizeof(double2) * d.px, st>>>(d, Z);
    k64_cols<<<ncols, 256, sizeof(double2) * d.py, st>>>(d_dev, cols, Z, nullptr, 1, 1);
    k64_response<<<nblocks(n), 256, 0, st>>>(d, Z, H, Hn, ramp ? 1 : 0);
}
void launch64_udm_admm(const SliceDesc* d, const BlockMap& rays, int nr, const double4_32a* t64, int ne,
                       const float4* meas, const F64Vecs& v, uint8_t* status, const SliceScalars* sc, int iters,
                       double* partial, cudaStream_t st) {
    k64_udm_admm<<<nr, 256, sizeof(double4_32a) * ne, st>>>(d, rays, t64, ne, meas, v.Rx, v.ua, v.a, v.mu, status, sc,
                                                        iters, partial);
}
void launch64_udm_init(const SliceDesc* d, const BlockMap& rays, int nr, const double4_32a* t64, int ne,
                       const float4* meas, const F64Vecs& v, double rho_p, int iters, double abar, double mu0,
                       cudaStream_t st) {
    k64_udm_init<<<nr, 256, sizeof(double4_32a) * ne, st>>>(d, rays, t64, ne, meas, v.a, v.mu, rho_p, iters, abar, mu0);
}
void launch64_image_update(const SliceDesc* d, const BlockMap& pix, int np, const SliceScalars* sc, double lam_c,
                           double lam_p, const F64Vecs& v, double* partial, cudaStream_t st) {
    k64_image_update<<<np, 256, 0, st>>>(d, pix, sc, lam_c, lam_p, v.x, v.y, v.uy, v.z, v.uz, partial);
}
void launch64_dual_rescale(const SliceDesc* d, const BlockMap& pix, int np, const BlockMap& rays, int nr,
                           const SliceScalars* sc, const F64Vecs& v, cudaStream_t st) {
    k64_dual_rescale<<<np + nr, 256, 0, st>>>(d, pix, np, rays, sc, v.uy, v.uz, v.ua);
}
void launch64_init_image(const SliceDesc* d, const BlockMap& pix, int np, const int* has_x0, const F64Vecs& v,
                         double kappa, cudaStream_t st) {
    k64_init_image<<<np, 256, 0, st>>>(d, pix, has_x0, v.x0, v.x, kappa);
}
void launch64_state_from_image(const SliceDesc* d, const BlockMap& pix, int np, const BlockMap& rays, int nr,
                               const F64Vecs& v, double mu0, cudaStream_t st) {
    k64_state_from_image<<<np + nr, 256, 0, st>>>(d, pix, np, rays, v.x, v.y, v.uy, v.z, v.uz, v.Rx, v.a, v.ua, v.mu,
                                                  mu0);
}
void launch64_xi_partials(const SliceDesc* d, const BlockMap& pix, int np, const double* x, const float2* truth,
                          double* partial, cudaStream_t st) {
    k64_xi_partials<<<np, 256, 0, st>>>(d, pix, x, truth, partial);
}
void launch64_objective(const SliceDesc* d, const BlockMap& rays, int nr, const BlockMap& pix, int np,
                        const double4_32a* t64, int ne, const float4* meas, const double* q, const double* x,
                        double lam_c, double lam_p, double* part_rays, double* part_pix, cudaStream_t st) {
    k64_objective_rays<<<nr, 256, sizeof(double4_32a) * ne, st>>>(d, rays, t64, ne, meas, q, part_rays);
    k64_objective_tv<<<np, 256, 0, st>>>(d, pix, x, lam_c, lam_p, part_pix);
}
void launch64_from_f32(const float* in, int64_t n, double* out, cudaStream_t st) {
    if (n > 0) k64_from_f32<<<nblocks(2 * n), 256, 0, st>>>(in, n, out);
}

}  // namespace dect
