// Per-ray dual-energy decomposition, Eq. 13 (the "UDM" subproblem of the
// splitting scheme, Sec. 3.3), by Levenberg-Marquardt.
//
// One thread per ray; the spectral tables sit in shared memory and every
// lane reads the same entry (broadcast). Per LM iteration the thread
// evaluates f_h, f_l and their Jacobian at a (one pass over the energies:
// one exp2 and six FMAs per bin) and f_h, f_l at the trial point a + delta
// (one exp2 and two FMAs per bin): the 4 evaluations of f of Table 1. Energy
// sums are float32 (compensated). Residuals come from the ratio of a spectral
// sum to the measured transmission t = e^{-m}: f - m = -log(s / t), from
// log1p of the relative difference when s and t are within a factor 2, which
// keeps the float32 sum's accuracy without a float64 log; the cost change of
// the trial step is formed from the residual changes -log(s' / s), so the
// accept test (cost decreased) does not subtract two large costs. The 2x2
// Marquardt solve is float32 from the Jacobian's minors (see lm_ray), which
// keeps it consistent with its float32 inputs; no float64 in the LM loop
// (float64 throughput is low on this GPU).
#include <cuda_runtime.h>
#include <math.h>

#include "dect_internal.cuh"
#include "prec.cuh"
#include "reduce.cuh"
#include "f32x2.cuh"

namespace dect {

// One ray's inputs; v = (R x - u^a) is carried as an unevaluated sum hi + lo (exact in float32)
struct RayIn {
    float mh, ml, wh, wl;
    float vc_hi, vc_lo, vp_hi, vp_lo;
    float rc, rp;
};

// v = a - b as hi + lo with hi = fl(a - b) and lo its exact rounding error (two-sum)
__device__ __forceinline__ void split_diff(float a, float b, float& hi, float& lo) {
    hi = a - b;
    const float bb = a - hi;
    lo = (a - (hi + bb)) + (bb - b);
}

struct LmState {
    float ac, ap, mu;
    uint8_t status;
};

// Compensated addition of a block partial into a running sum (Kahan): keeps the spectral sums,
// whose logs enter the LM accept test, accurate to a few float32 ulps of the exponentials.
__device__ __forceinline__ void kahan_add(float& sum, float& comp, float v) {
    const float y = v - comp;
    const float t = sum + y;
    comp = (t - sum) - y;
    sum = t;
}

// Energy bins by the spectra's supports (SpecDev): both spectra may be non-zero below n_both, only the
// longer one (the high spectrum if tail_high) in [n_both, n_end), neither from n_end on. Zero-weight
// terms are exact zeros, so skipping them leaves every sum bit for bit as it was; the compensated
// additions still run once per block of 8 bins over all ne bins, so the blocking is unchanged too.
// Blocks that lie wholly in one range run an unrolled body without per-bin tests.

// one bin's terms: W = 3 both spectra, 1 the high one only, 2 the low one only
template <int W>
__device__ __forceinline__ void bin_jac(const float4* __restrict__ t1, const float4* __restrict__ t2, int e, float ac,
                                        float ap, float& bh, float& bl, float& shc, float& shp, float& slc,
                                        float& slp) {
    const float4 a = t1[e];
    const float4 b = t2[e];
    const float t = exp2f(-fmaf(a.x, ac, a.y * ap));
    if (W & 1) {
        bh = fmaf(a.z, t, bh);
        shc = fmaf(b.x, t, shc);
        shp = fmaf(b.y, t, shp);
    }
    if (W & 2) {
        bl = fmaf(a.w, t, bl);
        slc = fmaf(b.z, t, slc);
        slp = fmaf(b.w, t, slp);
    }
}

// 2^x with rounding errors that average out: x = n + r, n = rint(x), r in [-1/2, 1/2] (exact), 2^r =
// e^(r ln 2) by its Taylor series to degree 8 (truncation below 2e-10 relative, under 0.01 of float32's
// half ulp) evaluated by Horner's rule with fused multiply-adds, then scaled by 2^n (ldexpf: exact,
// down to subnormals and zero). Round-to-nearest errors of the Horner steps carry no sign preference,
// whereas a fast exponential with a consistent half-ulp bias shifts every f(a) by ~3e-8; that bias is
// harmless in the decomposition but not in a sum of many squared residuals whose mean is non-zero
// (the objective of Eq. 4), which is where this one is used.
__device__ __forceinline__ float exp2_series(float x) {
    constexpr double L = 0.69314718055994530942;  // ln 2
    constexpr float c1 = (float)L, c2 = (float)(L * L / 2.0), c3 = (float)(L * L * L / 6.0),
                    c4 = (float)(L * L * L * L / 24.0), c5 = (float)(L * L * L * L * L / 120.0),
                    c6 = (float)(L * L * L * L * L * L / 720.0), c7 = (float)(L * L * L * L * L * L * L / 5040.0),
                    c8 = (float)(L * L * L * L * L * L * L * L / 40320.0);
    const float n = rintf(x);
    const float r = x - n;
    float p = fmaf(c8, r, c7);
    p = fmaf(p, r, c6);
    p = fmaf(p, r, c5);
    p = fmaf(p, r, c4);
    p = fmaf(p, r, c3);
    p = fmaf(p, r, c2);
    p = fmaf(p, r, c1);
    p = fmaf(p, r, 1.0f);
    return ldexpf(p, (int)fmaxf(n, -200.0f));
}

template <int W, bool SERIES = false>
__device__ __forceinline__ void bin_val(const float4* __restrict__ t1, int e, float ac, float ap, float& bh, float& bl) {
    const float4 a = t1[e];
    const float x = -fmaf(a.x, ac, a.y * ap);
    const float t = SERIES ? exp2_series(x) : exp2f(x);
    if (W & 1) bh = fmaf(a.z, t, bh);
    if (W & 2) bl = fmaf(a.w, t, bl);
}

// s_h, s_l (compensated, in blocks of 8 energies) and the four Jacobian numerators at (ac, ap).
__device__ __forceinline__ void spectral_sums_jac(const float4* __restrict__ t1, const float4* __restrict__ t2,
                                                  const SpecDev& sp, float ac, float ap, float& sh, float& sl,
                                                  float& shc, float& shp, float& slc, float& slp) {
    float ch = 0.f, cl = 0.f;
    sh = sl = shc = shp = slc = slp = 0.f;
    for (int e0 = 0; e0 < sp.ne; e0 += 8) {
        float bh = 0.f, bl = 0.f;
        if (e0 + 8 <= sp.n_both) {
            // both spectra: the sum pairs {b_h, b_l}, {s_hc, s_hp}, {s_lc, s_lp} advance as packed float32
            // pairs, each sum taking bin_jac<3>'s terms in its order (the same bits, half the instructions)
            f32x2 bhl = pack2(0.f, 0.f), sh2 = pack2(shc, shp), sl2 = pack2(slc, slp);
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const float4 a = t1[e0 + u];
                const float4 b = t2[e0 + u];
                const float t = exp2f(-fmaf(a.x, ac, a.y * ap));
                const f32x2 tt = pack2(t, t);
                bhl = fma2(pack2(a.z, a.w), tt, bhl);
                sh2 = fma2(pack2(b.x, b.y), tt, sh2);
                sl2 = fma2(pack2(b.z, b.w), tt, sl2);
            }
            const float2 x = unpack2(bhl), y = unpack2(sh2), z = unpack2(sl2);
            bh = x.x;
            bl = x.y;
            shc = y.x;
            shp = y.y;
            slc = z.x;
            slp = z.y;
        } else if (e0 >= sp.n_both && e0 + 8 <= sp.n_end) {
            if (sp.tail_high) {
#pragma unroll
                for (int u = 0; u < 8; ++u) bin_jac<1>(t1, t2, e0 + u, ac, ap, bh, bl, shc, shp, slc, slp);
            } else {
#pragma unroll
                for (int u = 0; u < 8; ++u) bin_jac<2>(t1, t2, e0 + u, ac, ap, bh, bl, shc, shp, slc, slp);
            }
        } else {
            const int e1 = min(e0 + 8, sp.n_end);
            for (int e = e0; e < e1; ++e) {
                if (e < sp.n_both)
                    bin_jac<3>(t1, t2, e, ac, ap, bh, bl, shc, shp, slc, slp);
                else if (sp.tail_high)
                    bin_jac<1>(t1, t2, e, ac, ap, bh, bl, shc, shp, slc, slp);
                else
                    bin_jac<2>(t1, t2, e, ac, ap, bh, bl, shc, shp, slc, slp);
            }
        }
        kahan_add(sh, ch, bh);
        kahan_add(sl, cl, bl);
    }
}

template <bool SERIES = false>
__device__ __forceinline__ void spectral_sums(const float4* __restrict__ t1, const SpecDev& sp, float ac, float ap,
                                              float& sh, float& sl) {
    float ch = 0.f, cl = 0.f;
    sh = sl = 0.f;
    for (int e0 = 0; e0 < sp.ne; e0 += 8) {
        float bh = 0.f, bl = 0.f;
        if (e0 + 8 <= sp.n_both) {
#pragma unroll
            for (int u = 0; u < 8; ++u) bin_val<3, SERIES>(t1, e0 + u, ac, ap, bh, bl);
        } else if (e0 >= sp.n_both && e0 + 8 <= sp.n_end) {
            if (sp.tail_high) {
#pragma unroll
                for (int u = 0; u < 8; ++u) bin_val<1, SERIES>(t1, e0 + u, ac, ap, bh, bl);
            } else {
#pragma unroll
                for (int u = 0; u < 8; ++u) bin_val<2, SERIES>(t1, e0 + u, ac, ap, bh, bl);
            }
        } else {
            const int e1 = min(e0 + 8, sp.n_end);
            for (int e = e0; e < e1; ++e) {
                if (e < sp.n_both)
                    bin_val<3, SERIES>(t1, e, ac, ap, bh, bl);
                else if (sp.tail_high)
                    bin_val<1, SERIES>(t1, e, ac, ap, bh, bl);
                else
                    bin_val<2, SERIES>(t1, e, ac, ap, bh, bl);
            }
        }
        kahan_add(sh, ch, bh);
        kahan_add(sl, cl, bl);
    }
}

// -log(a / b) for positive a, b: from the relative difference when the ratio is within [1/2, 2] (then
// a - b is exact and log1p keeps its accuracy), from the ratio itself otherwise (photon-starved
// rays whose model sum is orders of magnitude off the measurement, large trial steps)
__device__ __forceinline__ float neg_log_ratio(float a, float b) {
    const float q = a / b;
    return (q > 0.5f && q < 2.0f) ? -log1pf((a - b) / b) : -logf(q);
}

// a * b - c * d with one rounding of the result (the rounding error of c * d is recovered by an fma)
__device__ __forceinline__ float diff_of_products(float a, float b, float c, float d) {
    const float w = c * d;
    const float e = fmaf(-c, d, w);
    return fmaf(a, b, -w) + e;
}

// `iters` LM iterations of Eq. 13 for one ray (tables t1/t2 in shared memory).
//
// The Marquardt-damped Gauss-Newton step solves B d = -g with B = J^T W J + diag(e) (W = diag(w_h, w_l),
// J the 2x2 Jacobian of f, e_b = rho_b + mu (B_bb of the undamped matrix)) and g = J^T W r + q,
// q = rho (a - v). For a 2x2 J these follow from J's minors (Cauchy-Binet):
//   det B   = w_h w_l det(J)^2 + e_0 C_11 + e_1 C_00 + e_0 e_1         (C = J^T W J; every term >= 0)
//   adj(B) g = w_h w_l det(J) adj(J) r + adj(J) diag(w_l, w_h) adj(J)^T q + (e_1 g_0, e_0 g_1)
// so the cancellations of nearly collinear Compton and photoelectric columns happen only inside
// det(J) and the adj(J) products, each one fma-compensated difference of products: the float32 solve
// stays consistent with its float32 Jacobian, like a float64 solve of the same inputs.
__device__ void lm_ray(const float4* __restrict__ t1, const float4* __restrict__ t2, const SpecDev& sp,
                       const RayIn& in, int iters, LmState& s) {
    const float tm_h = expf(-in.mh), tm_l = expf(-in.ml);
    const float wh = in.wh, wl = in.wl, rc = in.rc, rp = in.rp;
    for (int it = 0; it < iters; ++it) {
        float sh, sl, shc, shp, slc, slp;
        spectral_sums_jac(t1, t2, sp, s.ac, s.ap, sh, sl, shc, shp, slc, slp);
        const float rh = neg_log_ratio(sh, tm_h), rl = neg_log_ratio(sl, tm_l);  // f - m = -log(s / t)
        const float j0 = shc / sh, j1 = shp / sh, j2 = slc / sl, j3 = slp / sl;
        const float dc = (s.ac - in.vc_hi) - in.vc_lo, dp = (s.ap - in.vp_hi) - in.vp_lo;  // a - v
        const float q0 = rc * dc, q1 = rp * dp;
        const float C00 = fmaf(wh * j0, j0, wl * j2 * j2), C11 = fmaf(wh * j1, j1, wl * j3 * j3);
        const float e0 = fmaf(s.mu, C00 + rc, rc), e1 = fmaf(s.mu, C11 + rp, rp);
        const float dJ = diff_of_products(j0, j3, j1, j2);
        const float whl = wh * wl;
        const float det = fmaf(whl * dJ, dJ, fmaf(e0, C11, fmaf(e1, C00, e0 * e1)));
        if (!(det > 0.0f) || !isfinite(det) || !isfinite(rh) || !isfinite(rl)) {
            s.status = DECT_RAY_NONFINITE;
            break;
        }
        const float g0 = fmaf(wh * rh, j0, fmaf(wl * rl, j2, q0));
        const float g1 = fmaf(wh * rh, j1, fmaf(wl * rl, j3, q1));
        const float ar0 = diff_of_products(j3, rh, j1, rl), ar1 = diff_of_products(j0, rl, j2, rh);
        const float u0 = wl * diff_of_products(j3, q0, j2, q1), u1 = wh * diff_of_products(j0, q1, j1, q0);
        const float aq0 = diff_of_products(j3, u0, j1, u1), aq1 = diff_of_products(j0, u1, j2, u0);
        const float n0 = fmaf(whl * dJ, ar0, aq0) + e1 * g0;
        const float n1 = fmaf(whl * dJ, ar1, aq1) + e0 * g1;
        const float tc = s.ac - n0 / det, tp = s.ap - n1 / det;
        float th, tl;
        spectral_sums(t1, sp, tc, tp, th, tl);
        // 2 (cost(trial) - cost(a)) = sum_k w_k (r1 - r0)(r1 + r0) + sum_b rho_b e_b (e_b + 2 (a_b - v_b))
        const float eh = neg_log_ratio(th, sh), el = neg_log_ratio(tl, sl);  // r1 - r0
        const float ec = tc - s.ac, ep = tp - s.ap;
        const float dcost = (wh * eh * fmaf(2.0f, rh, eh) + wl * el * fmaf(2.0f, rl, el)) +
                            (rc * ec * fmaf(2.0f, dc, ec) + rp * ep * fmaf(2.0f, dp, ep));
        float mu = s.mu;
        if (!isfinite(dcost)) {
            mu *= 10.f;
            s.status = DECT_RAY_NONFINITE;
        } else if (dcost < 0.0f) {
            s.ac = tc;
            s.ap = tp;
            mu *= 0.1f;
            s.status = DECT_RAY_ACCEPTED;
        } else {
            mu *= 10.f;
            s.status = DECT_RAY_REJECTED;
        }
        s.mu = fminf(fmaxf(mu, 1e-10f), 1e10f);
    }
}

// ---- float64 decomposition arithmetic (dect_params.udm_f64 = 1) -------------------------------------
// The float32 exponentials of the kernel above, accumulated in float64 with float64 spectral weights
// (w1 = {S_h, S_l, S_h f_KN, S_h f_p}, w2 = {S_l f_KN, S_l f_p, -, -}); logs of the sums, the 2x2
// Marquardt solve and the accept test (a direct comparison of the Eq. 13 costs, as in the oracle) in
// float64. The exponent's argument is formed in float32 from the float32-rounded point.

__device__ __forceinline__ void spectral_sums64(const float4* __restrict__ t1, const double4_32a* __restrict__ w1,
                                                const double4_32a* __restrict__ w2, int ne, double ac, double ap,
                                                bool jac, double& fh, double& fl, double* J) {
    const float fa = (float)ac, fp = (float)ap;
    double sh = 0.0, sl = 0.0, shc = 0.0, shp = 0.0, slc = 0.0, slp = 0.0;
    for (int e = 0; e < ne; ++e) {
        const float4 a = t1[e];
        const double t = (double)exp2f(-fmaf(a.x, fa, a.y * fp));
        const double4_32a u = w1[e];
        sh = fma(u.x, t, sh);
        sl = fma(u.y, t, sl);
        if (jac) {
            const double4_32a v = w2[e];
            shc = fma(u.z, t, shc);
            shp = fma(u.w, t, shp);
            slc = fma(v.x, t, slc);
            slp = fma(v.y, t, slp);
        }
    }
    fh = -log(sh);
    fl = -log(sl);
    if (jac) {
        J[0] = shc / sh;
        J[1] = shp / sh;
        J[2] = slc / sl;
        J[3] = slp / sl;
    }
}

__device__ __forceinline__ double cost_f64(double fh, double fl, double mh, double ml, double wh, double wl, double ac,
                                           double ap, double vc, double vp, double rc, double rp) {
    const double rh = fh - mh, rl = fl - ml;
    return 0.5 * (wh * rh * rh + wl * rl * rl) + 0.5 * (rc * (ac - vc) * (ac - vc) + rp * (ap - vp) * (ap - vp));
}

__device__ void lm_ray64(const float4* __restrict__ t1, const double4_32a* __restrict__ w1, const double4_32a* __restrict__ w2,
                         int ne, const RayIn& in, int iters, LmState& s) {
    const double mh = in.mh, ml = in.ml, wh = in.wh, wl = in.wl, rc = in.rc, rp = in.rp;
    const double vc = (double)in.vc_hi + (double)in.vc_lo, vp = (double)in.vp_hi + (double)in.vp_lo;
    double a0 = s.ac, a1 = s.ap, m = s.mu;
    for (int it = 0; it < iters; ++it) {
        double fh, fl, J[4];
        spectral_sums64(t1, w1, w2, ne, a0, a1, true, fh, fl, J);
        const double rh = fh - mh, rl = fl - ml;
        const double g0 = wh * rh * J[0] + wl * rl * J[2] + rc * (a0 - vc);
        const double g1 = wh * rh * J[1] + wl * rl * J[3] + rp * (a1 - vp);
        const double A00 = wh * J[0] * J[0] + wl * J[2] * J[2] + rc;
        const double A01 = wh * J[0] * J[1] + wl * J[2] * J[3];
        const double A11 = wh * J[1] * J[1] + wl * J[3] * J[3] + rp;
        const double B00 = A00 * (1.0 + m), B11 = A11 * (1.0 + m);
        const double det = B00 * B11 - A01 * A01;
        const double cost0 = cost_f64(fh, fl, mh, ml, wh, wl, a0, a1, vc, vp, rc, rp);
        if (!(det > 0.0) || !isfinite(det) || !isfinite(cost0)) {
            s.status = DECT_RAY_NONFINITE;
            break;
        }
        const double t0 = a0 + (-g0 * B11 + g1 * A01) / det;
        const double t1_ = a1 + (-g1 * B00 + g0 * A01) / det;
        double fh1, fl1;
        spectral_sums64(t1, w1, w2, ne, t0, t1_, false, fh1, fl1, nullptr);
        const double cost1 = cost_f64(fh1, fl1, mh, ml, wh, wl, t0, t1_, vc, vp, rc, rp);
        if (!isfinite(cost1)) {
            m *= 10.0;
            s.status = DECT_RAY_NONFINITE;
        } else if (cost1 < cost0) {
            a0 = t0;
            a1 = t1_;
            m /= 10.0;
            s.status = DECT_RAY_ACCEPTED;
        } else {
            m *= 10.0;
            s.status = DECT_RAY_REJECTED;
        }
        m = fmin(fmax(m, 1e-10), 1e10);
    }
    s.ac = (float)a0;
    s.ap = (float)a1;
    s.mu = (float)m;
}

__device__ __forceinline__ void load_tables(const SpecDev& sp, float4* t1, float4* t2) {
    for (int e = threadIdx.x; e < sp.ne; e += blockDim.x) {
        t1[e] = __ldg(sp.t1 + e);
        t2[e] = __ldg(sp.t2 + e);
    }
    __syncthreads();
}

// ADMM a-update fused with the a-block of the dual update (Eq. 11) and the a-block residual sums:
// partial[4*blk + {0,1}] = sum (a - Rx)^2 (c, p); partial[4*blk + {2,3}] = sum (a - a_old)^2.
template <class S2, bool F64>
__global__ void __launch_bounds__(kRaysPerBlock) k_udm_admm(const SliceDesc* __restrict__ dsl, BlockMap map, SpecDev sp,
                                                            const float4* __restrict__ meas,
                                                            const S2* __restrict__ Rx, S2* __restrict__ ua,
                                                            S2* __restrict__ a, float* __restrict__ mu,
                                                            uint8_t* __restrict__ status,
                                                            const SliceScalars* __restrict__ sc, int iters,
                                                            double* __restrict__ partial) {
    extern __shared__ float4 tabs[];
    float4* t1 = tabs;
    float4* t2 = tabs + sp.ne;
    double4_32a* w1 = reinterpret_cast<double4_32a*>(tabs + 2 * sp.ne);
    double4_32a* w2 = w1 + sp.ne;
    if (F64)
        for (int e = threadIdx.x; e < sp.ne; e += blockDim.x) {
            w1[e] = sp.w1[e];
            w2[e] = sp.w2[e];
        }
    load_tables(sp, t1, t2);
    int local;
    const int s = slice_of(map, blockIdx.x, local);
    const SliceDesc& d = dsl[s];
    const int64_t n = (int64_t)d.g.nv * d.g.nb;
    const int64_t r = (int64_t)local * kRaysPerBlock + threadIdx.x;
    float acc[4] = {0.f, 0.f, 0.f, 0.f};
    if (r < n) {
        const int64_t e = d.sino_off + r;
        const float4 m = __ldg(meas + e);
        const float2 rx = ldg2(Rx + e);
        float2 u = ld2(ua + e);
        const float2 a_old = ld2(a + e);
        RayIn in;
        in.mh = m.x;
        in.ml = m.y;
        in.wh = m.z;
        in.wl = m.w;
        split_diff(rx.x, u.x, in.vc_hi, in.vc_lo);
        split_diff(rx.y, u.y, in.vp_hi, in.vp_lo);
        in.rc = sc[s].rho_f[0];
        in.rp = sc[s].rho_f[1];
        LmState st{a_old.x, a_old.y, mu[e], DECT_RAY_ACCEPTED};
        if (F64)
            lm_ray64(t1, w1, w2, sp.ne, in, iters, st);
        else
            lm_ray(t1, t2, sp, in, iters, st);
        // the stored (possibly rounded) a is what the dual update and the residuals see
        st2(a + e, make_float2(st.ac, st.ap));
        const float2 an = ld2(a + e);
        mu[e] = st.mu;
        if (status) status[e] = st.status;
        const float rc = an.x - rx.x, rp = an.y - rx.y;
        u.x += rc;
        u.y += rp;
        st2(ua + e, u);
        const float dc = an.x - a_old.x, dp = an.y - a_old.y;
        acc[0] = rc * rc;
        acc[1] = rp * rp;
        acc[2] = dc * dc;
        acc[3] = dp * dp;
    }
    block_partials<4>(acc, partial);
}

// Initial decomposition: rho = (0, rho_p), v = 0, from a = (m_l / abar, 0), mu = mu0.
template <class S2>
__global__ void __launch_bounds__(kRaysPerBlock) k_udm_init(const SliceDesc* __restrict__ dsl, BlockMap map, SpecDev sp,
                                                            const float4* __restrict__ meas, S2* __restrict__ a,
                                                            float* __restrict__ mu, double rho_p, int iters,
                                                            float abar, float mu0) {
    extern __shared__ float4 tabs[];
    float4* t1 = tabs;
    float4* t2 = tabs + sp.ne;
    load_tables(sp, t1, t2);
    int local;
    const int s = slice_of(map, blockIdx.x, local);
    const SliceDesc& d = dsl[s];
    const int64_t n = (int64_t)d.g.nv * d.g.nb;
    const int64_t r = (int64_t)local * kRaysPerBlock + threadIdx.x;
    if (r >= n) return;
    const int64_t e = d.sino_off + r;
    const float4 m = __ldg(meas + e);
    RayIn in;
    in.mh = m.x;
    in.ml = m.y;
    in.wh = m.z;
    in.wl = m.w;
    in.vc_hi = in.vc_lo = in.vp_hi = in.vp_lo = 0.0f;
    in.rc = 0.0f;
    in.rp = (float)rho_p;
    LmState st{m.y / abar, 0.0f, mu0, DECT_RAY_ACCEPTED};
    lm_ray(t1, t2, sp, in, iters, st);
    st2(a + e, make_float2(st.ac, 0.0f));
    mu[e] = mu0;
}

// Public per-ray entry point (planar float arrays).
__global__ void __launch_bounds__(kRaysPerBlock) k_udm_rays(SpecDev sp, int64_t n, const float* __restrict__ mh,
                                                            const float* __restrict__ ml, const float* __restrict__ wh,
                                                            const float* __restrict__ wl, const float* __restrict__ vc,
                                                            const float* __restrict__ vp, double rho_c, double rho_p,
                                                            int iters, float* __restrict__ ac, float* __restrict__ ap,
                                                            float* __restrict__ mu, uint8_t* __restrict__ status) {
    extern __shared__ float4 tabs[];
    float4* t1 = tabs;
    float4* t2 = tabs + sp.ne;
    load_tables(sp, t1, t2);
    const int64_t r = (int64_t)blockIdx.x * kRaysPerBlock + threadIdx.x;
    if (r >= n) return;
    RayIn in;
    in.mh = __ldg(mh + r);
    in.ml = __ldg(ml + r);
    in.wh = __ldg(wh + r);
    in.wl = __ldg(wl + r);
    in.vc_hi = __ldg(vc + r);
    in.vp_hi = __ldg(vp + r);
    in.vc_lo = in.vp_lo = 0.0f;
    in.rc = (float)rho_c;
    in.rp = (float)rho_p;
    LmState st{ac[r], ap[r], mu[r], DECT_RAY_ACCEPTED};
    lm_ray(t1, t2, sp, in, iters, st);
    ac[r] = st.ac;
    ap[r] = st.ap;
    mu[r] = st.mu;
    if (status) status[r] = st.status;
}

// ---- comparison scheme LM(m) x CG(n): the per-ray parts of one LM step on basis b --------------------

// Gauss-Newton weights at the current projections: e = w_h r_h J_h,b + w_l r_l J_l,b and
// g = w_h J_h,b^2 + w_l J_l,b^2 (r = f - m), the spectral sums s0 = {s_h, s_l} for the trial's cost
// change, and R d cleared.
__global__ void __launch_bounds__(kRaysPerBlock) k_lm_rays(const SliceDesc* __restrict__ dsl, BlockMap map, SpecDev sp,
                                                           const float4* __restrict__ meas,
                                                           const float2* __restrict__ Rx, int b, float* __restrict__ ew,
                                                           float* __restrict__ gw, float2* __restrict__ s0,
                                                           float* __restrict__ Rd) {
    extern __shared__ float4 tabs[];
    float4* t1 = tabs;
    float4* t2 = tabs + sp.ne;
    load_tables(sp, t1, t2);
    int local;
    const int s = slice_of(map, blockIdx.x, local);
    const SliceDesc& d = dsl[s];
    const int64_t r = (int64_t)local * kRaysPerBlock + threadIdx.x;
    if (r >= (int64_t)d.g.nv * d.g.nb) return;
    const int64_t e = d.sino_off + r;
    const float4 m = __ldg(meas + e);
    const float2 a = __ldg(Rx + e);
    float sh, sl, shc, shp, slc, slp;
    spectral_sums_jac(t1, t2, sp, a.x, a.y, sh, sl, shc, shp, slc, slp);
    const float rh = neg_log_ratio(sh, expf(-m.x)), rl = neg_log_ratio(sl, expf(-m.y));
    const float jh = (b ? shp : shc) / sh, jl = (b ? slp : slc) / sl;
    ew[e] = m.z * rh * jh + m.w * rl * jl;
    gw[e] = m.z * jh * jh + m.w * jl * jl;
    s0[e] = make_float2(sh, sl);
    Rd[e] = 0.f;
}

// Change of the data term 1/2 sum_k w_k r_k^2 when basis b's projections move by R d:
// 1/2 sum_k w_k (r1 - r0)(r1 + r0) with r1 - r0 = -log(s1 / s0); partial[blk] = sum.
__global__ void __launch_bounds__(kRaysPerBlock) k_lm_trial(const SliceDesc* __restrict__ dsl, BlockMap map,
                                                            SpecDev sp, const float4* __restrict__ meas,
                                                            const float2* __restrict__ Rx, int b,
                                                            const float* __restrict__ Rd,
                                                            const float2* __restrict__ s0,
                                                            double* __restrict__ partial) {
    extern __shared__ float4 tabs[];
    float4* t1 = tabs;
    float4* t2 = tabs + sp.ne;
    load_tables(sp, t1, t2);
    int local;
    const int s = slice_of(map, blockIdx.x, local);
    const SliceDesc& d = dsl[s];
    const int64_t r = (int64_t)local * kRaysPerBlock + threadIdx.x;
    double acc[1] = {0.0};
    if (r < (int64_t)d.g.nv * d.g.nb) {
        const int64_t e = d.sino_off + r;
        const float4 m = __ldg(meas + e);
        float2 a = __ldg(Rx + e);
        if (b) a.y += __ldg(Rd + e); else a.x += __ldg(Rd + e);
        float sh, sl;
        spectral_sums(t1, sp, a.x, a.y, sh, sl);
        const float2 o = __ldg(s0 + e);
        const float r0h = neg_log_ratio(o.x, expf(-m.x)), r0l = neg_log_ratio(o.y, expf(-m.y));
        const float eh = neg_log_ratio(sh, o.x), el = neg_log_ratio(sl, o.y);
        acc[0] = 0.5 * ((double)m.z * eh * (2.0 * r0h + eh) + (double)m.w * el * (2.0 * r0l + el));
    }
    block_partials<1>(acc, partial);
}

static size_t tab_bytes(const SpecDev& sp) { return 2 * sizeof(float4) * (size_t)sp.ne; }
// ---- Eq. 4's data term, per ray -------------------------------------------------------------------

// partial[blk] = sum over the block's rays of 1/2 (w_h r_h^2 + w_l r_l^2), r = f(q) - m at the
// projections q = R x (stored in S2), with the spectral sums and residuals of the decomposition.
template <class S2>
__global__ void __launch_bounds__(kRaysPerBlock) k_objective_rays(const SliceDesc* __restrict__ dsl, BlockMap map,
                                                                  SpecDev sp, const float4* __restrict__ meas,
                                                                  const S2* __restrict__ q,
                                                                  double* __restrict__ partial) {
    extern __shared__ float4 tabs[];
    float4* t1 = tabs;
    float4* t2 = tabs + sp.ne;
    load_tables(sp, t1, t2);
    int local;
    const SliceDesc& d = dsl[slice_of(map, blockIdx.x, local)];
    const int64_t r = (int64_t)local * kRaysPerBlock + threadIdx.x;
    double acc[1] = {0.0};
    if (r < (int64_t)d.g.nv * d.g.nb) {
        const int64_t e = d.sino_off + r;
        const float4 m = __ldg(meas + e);
        const float2 a = ldg2(q + e);
        float sh, sl;
        spectral_sums<true>(t1, sp, a.x, a.y, sh, sl);
        // r = f - m = -log(s) - m in float64 from the float32 sum (the sum carries ~1 ulp, without bias)
        const double rh = -log((double)sh) - (double)m.x, rl = -log((double)sl) - (double)m.y;
        acc[0] = 0.5 * ((double)m.z * rh * rh + (double)m.w * rl * rl);
    }
    block_partials<1>(acc, partial);
}



void launch_lm_rays(const SliceDesc* dsl, const BlockMap& map, int nblk, const SpecDev& sp, const float4* meas,
                    const float2* Rx, int b, float* ew, float* gw, float2* s0, float* Rd, cudaStream_t st) {
    k_lm_rays<<<nblk, kRaysPerBlock, tab_bytes(sp), st>>>(dsl, map, sp, meas, Rx, b, ew, gw, s0, Rd);
}
void launch_lm_trial(const SliceDesc* dsl, const BlockMap& map, int nblk, const SpecDev& sp, const float4* meas,
                     const float2* Rx, int b, const float* Rd, const float2* s0, double* partial, cudaStream_t st) {
    k_lm_trial<<<nblk, kRaysPerBlock, tab_bytes(sp), st>>>(dsl, map, sp, meas, Rx, b, Rd, s0, partial);
}

// ---- forward model f (Eq. 3) and its Jacobian-transpose product, per ray ---------------------------
// float32: the LM kernel's sums (compensated, float32 exponentials), logs and ratios in float64.
// float64: tables and exponentials in float64 (t64 = {S_h, S_l, f_KN, f_p} per energy, unit-sum S).

__global__ void __launch_bounds__(kRaysPerBlock) k_forward_model_f32(SpecDev sp, int64_t n, const float* __restrict__ ac,
                                                                     const float* __restrict__ ap, float* __restrict__ fh,
                                                                     float* __restrict__ fl, float* __restrict__ jac,
                                                                     const float* __restrict__ gh,
                                                                     const float* __restrict__ gl, float* __restrict__ oc,
                                                                     float* __restrict__ op) {
    extern __shared__ float4 tabs[];
    float4* t1 = tabs;
    float4* t2 = tabs + sp.ne;
    load_tables(sp, t1, t2);
    const int64_t r = (int64_t)blockIdx.x * kRaysPerBlock + threadIdx.x;
    if (r >= n) return;
    float sh, sl, shc, shp, slc, slp;
    spectral_sums_jac(t1, t2, sp, __ldg(ac + r), __ldg(ap + r), sh, sl, shc, shp, slc, slp);
    const double ish = 1.0 / (double)sh, isl = 1.0 / (double)sl;
    const double j0 = shc * ish, j1 = shp * ish, j2 = slc * isl, j3 = slp * isl;
    if (fh) fh[r] = (float)(-log((double)sh));
    if (fl) fl[r] = (float)(-log((double)sl));
    if (jac) {
        jac[4 * r] = (float)j0;
        jac[4 * r + 1] = (float)j1;
        jac[4 * r + 2] = (float)j2;
        jac[4 * r + 3] = (float)j3;
    }
    if (oc) {
        const double a = __ldg(gh + r), b = __ldg(gl + r);
        oc[r] = (float)(a * j0 + b * j2);
        op[r] = (float)(a * j1 + b * j3);
    }
}

__global__ void __launch_bounds__(kRaysPerBlock) k_forward_model_f64(int ne, const double4_32a* __restrict__ t64, int64_t n,
                                                                     const double* __restrict__ ac,
                                                                     const double* __restrict__ ap, double* __restrict__ fh,
                                                                     double* __restrict__ fl, double* __restrict__ jac,
                                                                     const double* __restrict__ gh,
                                                                     const double* __restrict__ gl,
                                                                     double* __restrict__ oc, double* __restrict__ op) {
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    const double c = ac[r], p = ap[r];
    double sh = 0, sl = 0, shc = 0, shp = 0, slc = 0, slp = 0;
    for (int e = 0; e < ne; ++e) {
        const double4_32a T = t64[e];  // {S_h, S_l, f_KN, f_p}
        const double t = exp(-T.z * c - T.w * p);
        sh += T.x * t;
        sl += T.y * t;
        shc += T.x * T.z * t;
        shp += T.x * T.w * t;
        slc += T.y * T.z * t;
        slp += T.y * T.w * t;
    }
    const double j0 = shc / sh, j1 = shp / sh, j2 = slc / sl, j3 = slp / sl;
    if (fh) fh[r] = -log(sh);
    if (fl) fl[r] = -log(sl);
    if (jac) {
        jac[4 * r] = j0;
        jac[4 * r + 1] = j1;
        jac[4 * r + 2] = j2;
        jac[4 * r + 3] = j3;
    }
    if (oc) {
        oc[r] = gh[r] * j0 + gl[r] * j2;
        op[r] = gh[r] * j1 + gl[r] * j3;
    }
}


void launch_forward_model(const SpecDev& sp, const double4_32a* t64, int64_t n, int dtype, const void* ac,
                          const void* ap, void* fh, void* fl, void* jac, const void* gh, const void* gl, void* oc,
                          void* op, cudaStream_t st) {
    if (n <= 0) return;
    if (dtype == DECT_F32)
        k_forward_model_f32<<<(unsigned)((n + kRaysPerBlock - 1) / kRaysPerBlock), kRaysPerBlock, tab_bytes(sp), st>>>(
            sp, n, (const float*)ac, (const float*)ap, (float*)fh, (float*)fl, (float*)jac, (const float*)gh,
            (const float*)gl, (float*)oc, (float*)op);
    else
        k_forward_model_f64<<<(unsigned)((n + 127) / 128), 128, 0, st>>>(
            sp.ne, t64, n, (const double*)ac, (const double*)ap, (double*)fh, (double*)fl, (double*)jac,
            (const double*)gh, (const double*)gl, (double*)oc, (double*)op);
}

template <bool F64>
static void udm_admm_t(const SliceDesc* dsl, const BlockMap& map, int nblk, const SpecDev& sp, const float4* meas,
                       const void* Rx, void* ua, void* a, float* mu, uint8_t* status, const SliceScalars* sc,
                       int iters, double* partial, int prec, cudaStream_t st) {
    const size_t smem = tab_bytes(sp) + (F64 ? 2 * sizeof(double4_32a) * (size_t)sp.ne : 0);
    if (prec == PREC_F16)
        k_udm_admm<__half2, F64><<<nblk, kRaysPerBlock, smem, st>>>(
            dsl, map, sp, meas, (const __half2*)Rx, (__half2*)ua, (__half2*)a, mu, status, sc, iters, partial);
    else if (prec == PREC_BF16)
        k_udm_admm<__nv_bfloat162, F64><<<nblk, kRaysPerBlock, smem, st>>>(
            dsl, map, sp, meas, (const __nv_bfloat162*)Rx, (__nv_bfloat162*)ua, (__nv_bfloat162*)a, mu, status, sc,
            iters, partial);
    else
        k_udm_admm<float2, F64><<<nblk, kRaysPerBlock, smem, st>>>(
            dsl, map, sp, meas, (const float2*)Rx, (float2*)ua, (float2*)a, mu, status, sc, iters, partial);
}

void launch_udm_admm(const SliceDesc* dsl, const BlockMap& map, int nblk, const SpecDev& sp, const float4* meas,
                     const void* Rx, void* ua, void* a, float* mu, uint8_t* status, const SliceScalars* sc,
                     int iters, double* partial, int prec, bool f64, cudaStream_t st) {
    if (f64)
        udm_admm_t<true>(dsl, map, nblk, sp, meas, Rx, ua, a, mu, status, sc, iters, partial, prec, st);
    else
        udm_admm_t<false>(dsl, map, nblk, sp, meas, Rx, ua, a, mu, status, sc, iters, partial, prec, st);
}

void launch_objective_rays(const SliceDesc* dsl, const BlockMap& map, int nblk, const SpecDev& sp, const float4* meas,
                           const void* q, double* partial, int prec, cudaStream_t st) {
    if (prec == PREC_F16)
        k_objective_rays<__half2><<<nblk, kRaysPerBlock, tab_bytes(sp), st>>>(dsl, map, sp, meas, (const __half2*)q,
                                                                                partial);
    else if (prec == PREC_BF16)
        k_objective_rays<__nv_bfloat162><<<nblk, kRaysPerBlock, tab_bytes(sp), st>>>(
            dsl, map, sp, meas, (const __nv_bfloat162*)q, partial);
    else
        k_objective_rays<float2><<<nblk, kRaysPerBlock, tab_bytes(sp), st>>>(dsl, map, sp, meas, (const float2*)q,
                                                                               partial);
}

void launch_udm_init(const SliceDesc* dsl, const BlockMap& map, int nblk, const SpecDev& sp, const float4* meas,
                     void* a, float* mu, double rho_p, int iters, float abar, double mu0, int prec, cudaStream_t st) {
    if (prec == PREC_F16)
        k_udm_init<__half2><<<nblk, kRaysPerBlock, tab_bytes(sp), st>>>(dsl, map, sp, meas, (__half2*)a, mu, rho_p,
                                                                         iters, abar, (float)mu0);
    else if (prec == PREC_BF16)
        k_udm_init<__nv_bfloat162><<<nblk, kRaysPerBlock, tab_bytes(sp), st>>>(
            dsl, map, sp, meas, (__nv_bfloat162*)a, mu, rho_p, iters, abar, (float)mu0);
    else
        k_udm_init<float2><<<nblk, kRaysPerBlock, tab_bytes(sp), st>>>(dsl, map, sp, meas, (float2*)a, mu, rho_p,
                                                                        iters, abar, (float)mu0);
}

void launch_udm_rays(const SpecDev& sp, int64_t n, const float* mh, const float* ml, const float* wh, const float* wl,
                     const float* vc, const float* vp, double rho_c, double rho_p, int iters, float* ac, float* ap,
                     float* mu, uint8_t* status, cudaStream_t st) {
    if (n <= 0) return;
    k_udm_rays<<<(unsigned)((n + kRaysPerBlock - 1) / kRaysPerBlock), kRaysPerBlock, tab_bytes(sp), st>>>(
        sp, n, mh, ml, wh, wl, vc, vp, rho_c, rho_p, iters, ac, ap, mu, status);
}

}  // namespace dect
