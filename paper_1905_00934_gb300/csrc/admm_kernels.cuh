// Launchers of the element-wise / reduction kernels of one ADMM iteration (admm_kernels.cu).
#pragma once

#include "dect_internal.cuh"

namespace dect {

// (prec: storage format of the sinogram-domain vectors a, u^a, R x, q / b; see prec.cuh)
void launch_sino_resid(const SliceDesc* d, const BlockMap& rays, int nr, const void* a, const void* ua,
                       const void* Rx, void* b, int prec, cudaStream_t st);
void launch_rs_reduce(const double* part, const int* rows_prefix, SliceScalars* sc, int B, int first, cudaStream_t st);
void launch_alpha(const double* part, const int* bp_prefix, SliceScalars* sc, int B, cudaStream_t st);
void launch_cg_update(const SliceDesc* d, const BlockMap& pix, int np, const BlockMap& rays, int nr,
                      const SliceScalars* sc, float2* x, const float2* p, float2* r, const float2* Ap, void* Rx,
                      const void* q, int last, int prec, cudaStream_t st);
void launch_cg_p(const SliceDesc* d, const BlockMap& pix, int np, const SliceScalars* sc, const float2* s, float2* p,
                 cudaStream_t st);
void launch_image_update(const SliceDesc* d, const BlockMap& pix, int np, const SliceScalars* sc, double lam_c,
                         double lam_p, const float2* x, float4* y, float4* uy, float2* z, float2* uz, double* partial,
                         cudaStream_t st);
void launch_rho_update(const double* part_udm, const int* rays_prefix, const double* part_img, const int* pix_prefix,
                       SliceScalars* sc, int B, double mu_b, double tau, cudaStream_t st);
void launch_dual_rescale(const SliceDesc* d, int B, const SliceScalars* sc, float4* uy, float2* uz, void* ua, int prec,
                         cudaStream_t st);
void launch_xi(const SliceDesc* d, const BlockMap& pix, int np, const float2* x, const float2* truth, double* partial,
               SliceScalars* sc, int B, cudaStream_t st);
// Eq. 4's objective: TV partials per pixel block, then ray + pixel partials summed per slice into sc
void launch_objective_tv(const SliceDesc* d, const BlockMap& pix, int np, const float2* x, double lam_c, double lam_p,
                         double* partial, cudaStream_t st);
void launch_objective_reduce(const double* part_rays, const int* rays_prefix, const double* part_pix,
                             const int* pix_prefix, SliceScalars* sc, int B, cudaStream_t st);
// xi sums of the slices from per-pixel-block partials (4 per block) written by any xi partial kernel
void launch_xi_reduce(const double* partial, const int* pix_prefix, SliceScalars* sc, int B, cudaStream_t st);
void launch_init_image(const SliceDesc* d, const BlockMap& pix, int np, const int* has_x0, const float2* x0,
                       float2* x, float kappa, cudaStream_t st);
void launch_state_from_image(const SliceDesc* d, const BlockMap& pix, int np, const BlockMap& rays, int nr,
                             const float2* x, float4* y, float4* uy, float2* z, float2* uz, const void* Rx,
                             void* a, void* ua, float* mu, float mu0, int prec, cudaStream_t st);
void launch_reset_scalars(SliceScalars* sc, int B, double rho_c, double rho_p, cudaStream_t st);
void launch_pack_meas(const float* staged, int64_t n, float4* meas, cudaStream_t st);
void launch_interleave(const float* in, int64_t n, float2* out, cudaStream_t st);
void launch_deinterleave2(const void* in, int64_t n, float* out, int prec, cudaStream_t st);
void launch_deinterleave4(const float4* in, int64_t n, float* out, cudaStream_t st);

}  // namespace dect
