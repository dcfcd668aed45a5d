// Internal declarations of the dect library (GB300, sm_103a).
//
// Data layout in device memory
//  - Internal image vectors hold both bases interleaved: float2 {c, p} per
//    pixel, row-major [ny][nx]. The TV split variables y, u^y hold float4
//    {x-component c, y-component c, x-component p, y-component p}.
//  - Internal sinogram vectors are float2 {c, p} per ray, [n_views][n_bins].
//  - Measurements are float4 {m_h, m_l, w_h, w_l} per ray.
//  - The projector reads the image through two "pair textures" (plain global
//    arrays, no texture hardware): for rays sampled per column, TX[i][jj]
//    = {c(jj-2,i), p(jj-2,i), c(jj-1,i), p(jj-1,i)} for jj in [0, ny+2], zero
//    outside the image, so one 16-byte load gives both interpolation
//    neighbours of both bases; TY[j][ii] is the same along rows.
//  - Per-ray geometry table int4 {q0 low, q0 high, slope, +-w}: a ray with
//    w > 0 (axis 0) is sampled at every column i at fractional row
//    q0 + i * slope, q0 in 32.32 fixed point and slope in 2.30 fixed point,
//    and weighted by w = pixel/|d_x|; w < 0 (axis 1) swaps rows and columns.
//  - Batched solvers stack B slices in one allocation per array; a slice
//    descriptor holds each slice's offsets and geometry.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "../../include/dect.h"

namespace dect {

constexpr int kMaxEnergies = 512;
constexpr int kFftMaxLog2 = 12;  // padded FFT length up to 4096 per axis
constexpr int kFftMax = 1 << kFftMaxLog2;

// Geometry as the kernels see it (float copies for candidate searches).
struct GeomDev {
    int kind, nx, ny, nv, nb;
    float pix, du, uoff, sod, sdd;
    float cx, cy;           // (nx-1)/2, (ny-1)/2
    float inv_du;           // 1 / du
    float k0, k1;           // fractional bin of detector coordinate u: k = u * inv_du + k0; k1 = sdd * inv_du
    const int4* rays;       // [nv*nb] {q0 lo, q0 hi, slope, +-w}
    const float4* views;    // [nv] {cos, sin, axis layout: +-(s1 + 1), s2 or -1} (k_view_axes)
};

// One slice of a batched solver.
struct SliceDesc {
    GeomDev g;
    int64_t img_off;    // pixel offset (elements) in image arrays
    int64_t sino_off;   // ray offset in sinogram arrays
    int64_t tx_off;     // float4 offset in TX (nx*(ny+3) per slice)
    int64_t ty_off;     // float4 offset in TY (ny*(nx+3) per slice)
    int64_t fft_off;    // complex offset in the FFT work buffer (py*px per slice)
    int64_t h_off;      // float offset of the preconditioner response H [py][px]
    int32_t px, py, lpx, lpy;   // padded FFT sizes and their log2
};

// Maps a flat block index to (slice, block within slice) by a prefix table.
struct BlockMap {
    const int* prefix;  // device, B+1 entries
    int B;
};

__device__ __forceinline__ int slice_of(const BlockMap& m, int blk, int& local) {
    int lo = 0, hi = m.B - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (__ldg(m.prefix + mid) <= blk) lo = mid; else hi = mid - 1;
    }
    local = blk - __ldg(m.prefix + lo);
    return lo;
}

// Per-slice device scalars (CG, rho, residuals, monitors).
struct SliceScalars {
    double rho[2];
    double factor[2];    // rescale factor applied to the duals this iteration (1 = none)
    double rs[2];        // <r, M^-1 r>
    double alpha[2];
    double beta[2];
    double pAp[2];
    double r_pri[2];
    double r_dual[2];
    double xi_num[2], xi_den[2];
    // float32 copies for the element-wise kernels (float64 is slow on this GPU): CG step and direction
    // scalars, rho, and the factor the scaled duals are divided by this iteration
    float alpha_f[2], beta_f[2], rho_f[2], ifactor_f[2];
    int32_t iteration;
    int32_t objective_iter;  // the iteration the objective below was evaluated after (-1: never)
    double objective;        // Eq. 4 at that iteration's x
};

// Per-slice scalars of the comparison scheme LM(m) x CG(n) (one LM step on one basis at a time)
struct LmScalars {
    double mu[2];    // LM damping per basis (Marquardt scaling of the data curvature)
    double rr;       // CG: <r, r>
    double alpha;    // CG step
    double beta;     // CG direction update
    double dcost;    // change of the subproblem objective at the last trial point
    int32_t accept;  // the last trial step was accepted
    int32_t pad;
};

// Spectral tables on the device: T1 = {k_kn, k_p, S_h, S_l}, T2 = {S_h f_KN, S_h f_p, S_l f_KN, S_l f_p}
// with k = f * log2(e) so that exp(-f_KN a_c - f_p a_p) = exp2(-k_kn a_c - k_p a_p).
// w1 = {S_h, S_l, S_h f_KN, S_h f_p}, w2 = {S_l f_KN, S_l f_p, 0, 0} in float64 (unit-sum S), for the
// decomposition's float64 sums (dect_params.udm_f64).
// n_both, n_end, tail_high: the supports of the spectra (bins past a spectrum's last non-zero entry
// contribute exact zeros to its sums): both may be non-zero below n_both, only the high spectrum
// (tail_high) or only the low one in [n_both, n_end), neither from n_end on.
struct SpecDev {
    int ne;
    const float4* t1;
    const float4* t2;
    const double4_32a* w1;
    const double4_32a* w2;
    int n_both, n_end, tail_high;
};

// Epilogue modes of the backprojector.
enum BpMode {
    BP_PLAIN = 0,      // out = R^T s
    BP_R0 = 1,         // out = R^T b + D^T(y + u^y - D x) + (z + u^z - x)
    BP_AP = 2,         // out = R^T q + D^T D p + p, partial <p, out>
    BP_R0_NOGRAD = 3,  // out = R^T b + (z + u^z - x)
    BP_AP_NOGRAD = 4,  // out = R^T q + p, partial <p, out>
};

struct BpEpilogue {
    const float2* x;    // BP_R0*: current image
    const float4* y;
    const float4* uy;
    const float2* z;
    const float2* uz;
    const float2* p;    // BP_AP*: direction
    double* partial;    // BP_AP*: per-block {<p_c, Ap_c>, <p_p, Ap_p>}
};

// ---- launch helpers implemented in the .cu files ------------------------------------------

// projector.cu
cudaError_t build_ray_table(const dect_geom_desc& d, int4* rays, float4* views, cudaStream_t st);
// (prec: storage format of textures and sinogram vectors, see prec.cuh)
void launch_textures(const SliceDesc* dsl, const BlockMap& mx, int nbx, const BlockMap& my, int nby,
                     const float2* img, void* tx, void* ty, int prec, cudaStream_t st);
void launch_textures1(const SliceDesc* dsl, const BlockMap& mx, int nbx, const BlockMap& my, int nby,
                      const float* img, float2* tx, float2* ty, cudaStream_t st);
// projector CTAs (tiles of `views` views x 32 bins; views = 2, 4 or 8) of a slice; the projector's block
// maps count these per geometry group: up to proj_group_size() slices of one geometry, given as int4
// {slice, slices or -1}. The view count does not change results.
int proj_tiles(int nv, int nb, int views);
int proj_default_views();
int proj_group_size();
void launch_project1(const SliceDesc* dsl, const BlockMap& map, int nblk, const int4* groups, const float2* tx,
                     const float2* ty, float* out, int views, cudaStream_t st);
void launch_project(const SliceDesc* dsl, const BlockMap& map, int nblk, const int4* groups, const void* tx,
                    const void* ty, void* out, int prec, int views, cudaStream_t st);
// backproject_sweep.cu: the solver's backprojector (two kernels: sweep into C partial images, then
// the fixed-order sum of the partials with the epilogue; partial dots over the `pix` blocks)
int sweep_ctas_for_groups(int view_groups);
int sweep_groups_per_cta();
// image tiles of the sweep for a TILE x TILE tile (32 or 64); the occupancy choice of view groups
int sweep_tiles(int nx, int ny, int tile);
int sweep_groups(int tiles, int tile);
cudaError_t sweep_init_attributes();  // per device: dynamic shared memory of the 64-pixel tiles
constexpr int kSweepTileDefault = 32;
// cluster: the C view groups of a tile reduce on chip (thread-block cluster, distributed shared memory)
// into partial image 0 (the finalize pass then reads one image, C = 1); otherwise C partial images.
// sg = 2: the block map counts tiles of slice groups (groups: {slice, second slice or -1, -, -}) and a
// CTA backprojects into both slices of its group (plain form only); sg = 1: the map counts slices.
// tile_count (plain form, C >= 2; nullptr otherwise): one zeroed counter per tile of the launch
// (nsweep / C of them); the tile's last CTA sums the C partials into image 0 (the finalize pass then
// reads one image, C = 1) and zeroes the counter again.
void launch_bp_sweep(const SliceDesc* dsl, const BlockMap& smap, int nsweep, int C, int tile, bool cluster, int sg,
                     const int4* groups, const void* sino, float2* partial, int64_t stride, int prec, int* tile_count,
                     cudaStream_t st);
// single-channel sweep (float sinogram, float partial images; rw per ray and scale per slice optional)
void launch_bp_sweep1(const SliceDesc* dsl, const BlockMap& smap, int nsweep, int C, int tile, bool cluster,
                      const float* sino, const float* rw, const float* scale, float* partial, int64_t stride,
                      int* tile_count, cudaStream_t st);
void launch_bp_finalize(int mode, const SliceDesc* dsl, const BlockMap& pix, int npix, int C, const float2* partial,
                        int64_t stride, float2* out, const BpEpilogue& ep, cudaStream_t st);
// Single-slice planar R^T (dect_backproject): sino [nch][nv][nb] -> out [nch][ny][nx]. d_dev is the
// slice's descriptor on the device with zero offsets; maps holds the sweep and pixel-block prefixes
// {0, sweep_tiles * C, 0, pixel blocks}; packed holds nv*nb float2, partial C*nx*ny float2.
void backproject_single(const SliceDesc& sd, const SliceDesc* d_dev, const int* maps, int C, int tile, const float* sino,
                        int nch, float2* packed, float2* partial, float* out, cudaStream_t st);
void project_single(const SliceDesc& sd, const float* img, int nch, float2* scratch, float4* tx, float4* ty,
                    float* out, cudaStream_t st);
void launch_pack_planar(const float* in, int nch, int64_t n, float2* out, cudaStream_t st);
int texture_x_blocks(int nx, int ny);
int texture_y_blocks(int nx, int ny);
constexpr int kRaysPerBlock = 256;
constexpr int kPixPerBlock = 256;

// udm.cu
void launch_udm_admm(const SliceDesc* dsl, const BlockMap& map, int nblk, const SpecDev& sp, const float4* meas,
                     const void* Rx, void* ua, void* a, float* mu, uint8_t* status,
                     const SliceScalars* sc, int iters, double* partial, int prec, bool f64, cudaStream_t st);
// Eq. 4's data term: partial[blk] = sum 1/2 (w_h r_h^2 + w_l r_l^2) over the block's rays, r = f(q) - m
void launch_objective_rays(const SliceDesc* dsl, const BlockMap& map, int nblk, const SpecDev& sp, const float4* meas,
                           const void* q, double* partial, int prec, cudaStream_t st);
void launch_udm_init(const SliceDesc* dsl, const BlockMap& map, int nblk, const SpecDev& sp, const float4* meas,
                     void* a, float* mu, double rho_p, int iters, float abar, double mu0, int prec, cudaStream_t st);
void launch_udm_rays(const SpecDev& sp, int64_t n, const float* mh, const float* ml, const float* wh,
                     const float* wl, const float* vc, const float* vp, double rho_c, double rho_p, int iters,
                     float* ac, float* ap, float* mu, uint8_t* status, cudaStream_t st);

void launch_lm_rays(const SliceDesc* dsl, const BlockMap& map, int nblk, const SpecDev& sp, const float4* meas,
                    const float2* Rx, int b, float* ew, float* gw, float2* s0, float* Rd, cudaStream_t st);
void launch_lm_trial(const SliceDesc* dsl, const BlockMap& map, int nblk, const SpecDev& sp, const float4* meas,
                     const float2* Rx, int b, const float* Rd, const float2* s0, double* partial, cudaStream_t st);

// lmcg.cu
void launch_lm_reset(LmScalars* ls, int B, double mu0, cudaStream_t st);
void launch_lm_begin(const LmScalars* ls, float* scale, int B, int b, cudaStream_t st);
void launch_lm_grad(const SliceDesc* dsl, const BlockMap& pix, int npix, int C, const float* partial, int64_t stride,
                    int b, const SliceScalars* sc, const BpEpilogue& ep, float* r, float* p, float* dlt, double* part,
                    cudaStream_t st);
void launch_lm_ap(const SliceDesc* dsl, const BlockMap& pix, int npix, int C, const float* partial, int64_t stride,
                  int b, const SliceScalars* sc, const float* p, float* Ap, double* part, cudaStream_t st);
void launch_lm_alpha(const double* part, const int* prefix, LmScalars* ls, int B, cudaStream_t st);
void launch_lm_rr(const double* part, const int* prefix, LmScalars* ls, int B, int first, cudaStream_t st);
void launch_lm_cg(const SliceDesc* dsl, const BlockMap& pix, int npix, const BlockMap& rays, int nray,
                  const LmScalars* ls, float* dlt, const float* p, float* r, const float* Ap, float* Rd, const float* q,
                  int last, double* part, cudaStream_t st);
void launch_lm_p(const SliceDesc* dsl, const BlockMap& pix, int npix, const LmScalars* ls, const float* r, float* p,
                 cudaStream_t st);
void launch_lm_al_delta(const SliceDesc* dsl, const BlockMap& pix, int npix, int b, const SliceScalars* sc,
                        const BpEpilogue& ep, const float* dlt, double* part, cudaStream_t st);
void launch_lm_decide(const double* part_ray, const int* rays_prefix, const double* part_pix, const int* pix_prefix,
                      LmScalars* ls, float* scale, int B, int b, cudaStream_t st);
void launch_lm_accept(const SliceDesc* dsl, const BlockMap& pix, int npix, const BlockMap& rays, int nray,
                      const LmScalars* ls, int b, float2* x, const float* dlt, float2* Rx, const float* Rd,
                      cudaStream_t st);

void launch_forward_model(const SpecDev& sp, const double4_32a* t64, int64_t n, int dtype, const void* ac,
                          const void* ap, void* fh, void* fl, void* jac, const void* gh, const void* gl, void* oc,
                          void* op, cudaStream_t st);

// projector_f64.cu
cudaError_t build_ray_table_f64(const dect_geom_desc& d, double4_32a* rays, cudaStream_t st);
void project_single_f64(const GeomDev& g, const double4_32a* rays, const double* x, int nch, double* out, cudaStream_t st);
void backproject_single_f64(const GeomDev& g, const double4_32a* rays, const double* sino, int nch, double* out,
                            cudaStream_t st);

// fft.cu
const float2* fft_twiddles();   // device table exp(-2 pi i t / kFftMax), t < kFftMax/2 (current device)
__host__ __device__ int precond_cols_per_block(int py);
// The preconditioner's apply splits an axis of padded length p in 64..2048 into two half-length register
// FFTs (a pair of warps per row or column, 4 pairs per 256-thread block); other lengths take the staged
// path (one row, or precond_cols_per_block(py) columns, per block). The choice depends on the slice only.
__host__ __device__ inline bool precond_split(int p) { return p >= 64 && p <= 2048; }
inline int precond_rows_per_block(int px) { return precond_split(px) ? 4 : 1; }
inline int precond_apply_cols_per_block(int py) { return precond_split(py) ? 4 : precond_cols_per_block(py); }
// s = M^-1 r per slice and partial[2*blk] = <r, s> per channel over the row blocks
// (rows_map / cols_map: precond_rows_per_block / precond_apply_cols_per_block blocks; Hp: the response
// permuted for the split column pass, launch_permute_response)
void launch_precond(const SliceDesc* dsl, const BlockMap& rows_map, int nrows_blk, const BlockMap& cols_map,
                    int ncols_blk, const float* H, const float* Hp, const float2* r, float2* s, float2* Z,
                    double* partial_rs, const float2* tw, int max_px, int min_px, int max_py, int min_py,
                    cudaStream_t st);
// Hp[k][h py/2 + t] = H[2 bitrev(t) + h][frequency of storage column k], for a slice whose columns split
void launch_permute_response(const SliceDesc& d, const float* H, float* Hp, cudaStream_t st);
// H (and the variant without the D^T D term) from R^T R applied to a centred impulse (one slice)
// (d_dev: the slice's descriptor on the device with fft_off = h_off = 0; cols_map: its column groups)
void launch_psf_to_response(const SliceDesc* d_dev, const SliceDesc& d, const BlockMap& cols_map, int ncols,
                            const float2* psf, float2* Z, float* H, float* H_nograd, const float2* tw, bool ramp,
                            cudaStream_t st);
cudaError_t fft_init_attributes();

// ---- float64 solver path (solver_f64.cu) ----
// Device vectors of the float64 path, planar per slice: images [2][np] at 2 img_off, y / u^y
// [2][2][np] at 4 img_off, sinograms [2][nr] at 2 sino_off, mu [nr] at sino_off, Z at fft_off,
// H / Hn at h_off; RTs holds a backprojection [2][np] per slice.
struct F64Vecs {
    double *x = nullptr, *r = nullptr, *s = nullptr, *p = nullptr, *Ap = nullptr, *z = nullptr, *uz = nullptr;
    double *x0 = nullptr, *y = nullptr, *uy = nullptr, *RTs = nullptr;
    double *Rx = nullptr, *a = nullptr, *ua = nullptr, *q = nullptr, *mu = nullptr;
    double *H = nullptr, *Hn = nullptr;
    double2* Z = nullptr;
};
void launch64_sino_resid(const SliceDesc* d, const BlockMap& rays, int nr, const double* a, const double* ua,
                         const double* Rx, double* b, cudaStream_t st);
void launch64_r0(const SliceDesc* d, const BlockMap& pix, int np, const double* RTb, const F64Vecs& v, double* r,
                 bool with_grad, cudaStream_t st);
void launch64_ap(const SliceDesc* d, const BlockMap& pix, int np, const double* RTq, const double* p, double* Ap,
                 double* partial, bool with_grad, cudaStream_t st);
void launch64_cg_update(const SliceDesc* d, const BlockMap& pix, int np, const BlockMap& rays, int nr,
                        const SliceScalars* sc, const F64Vecs& v, int last, cudaStream_t st);
void launch64_cg_p(const SliceDesc* d, const BlockMap& pix, int np, const SliceScalars* sc, const double* s, double* p,
                   cudaStream_t st);
// s = M^-1 r (H null: plain CG, s = r); partial[2 row + c] = <r_c, s_c> over the image-row map
void launch64_precond(const SliceDesc* d, const BlockMap& rows, int nrows, const BlockMap& cols, int ncols,
                      const double* H, const double* r, double* s, double2* Z, double* partial, int max_px, int max_py,
                      cudaStream_t st);
void launch64_response(const SliceDesc* d_dev, const SliceDesc& d, const BlockMap& cols, int ncols, const double* psf,
                       double2* Z, double* H, double* Hn, bool ramp, cudaStream_t st);
void launch64_udm_admm(const SliceDesc* d, const BlockMap& rays, int nr, const double4_32a* t64, int ne,
                       const float4* meas, const F64Vecs& v, uint8_t* status, const SliceScalars* sc, int iters,
                       double* partial, cudaStream_t st);
void launch64_udm_init(const SliceDesc* d, const BlockMap& rays, int nr, const double4_32a* t64, int ne,
                       const float4* meas, const F64Vecs& v, double rho_p, int iters, double abar, double mu0,
                       cudaStream_t st);
void launch64_image_update(const SliceDesc* d, const BlockMap& pix, int np, const SliceScalars* sc, double lam_c,
                           double lam_p, const F64Vecs& v, double* partial, cudaStream_t st);
void launch64_dual_rescale(const SliceDesc* d, const BlockMap& pix, int np, const BlockMap& rays, int nr,
                           const SliceScalars* sc, const F64Vecs& v, cudaStream_t st);
void launch64_init_image(const SliceDesc* d, const BlockMap& pix, int np, const int* has_x0, const F64Vecs& v,
                         double kappa, cudaStream_t st);
void launch64_state_from_image(const SliceDesc* d, const BlockMap& pix, int np, const BlockMap& rays, int nr,
                               const F64Vecs& v, double mu0, cudaStream_t st);
void launch64_xi_partials(const SliceDesc* d, const BlockMap& pix, int np, const double* x, const float2* truth,
                          double* partial, cudaStream_t st);
void launch64_from_f32(const float* in, int64_t n, double* out, cudaStream_t st);
// Eq. 4's partials: data term per ray block at q = R x (part_rays), TV per pixel block (part_pix)
void launch64_objective(const SliceDesc* d, const BlockMap& rays, int nr, const BlockMap& pix, int np,
                        const double4_32a* t64, int ne, const float4* meas, const double* q, const double* x,
                        double lam_c, double lam_p, double* part_rays, double* part_pix, cudaStream_t st);

// ---- filtered backprojection and CDM-FBP (fbp.cu) ----
struct FbpDev {
    int nx, ny, nv, nb, fan;
    float pix, cx, cy;   // pixel pitch, image centre (pixels)
    float sod, k0, k1;   // fan: source distance; fractional bin k = k1 * (P.e) / den + k0 (k0 also in tab.z)
    float gain, scale;   // filter gain (1/du, or 1/(2 du SOD/SDD)); backprojection factor (pi/V, 2 pi/V)
    const float4* tab;   // [nv]: parallel {c/du, s/du, k0, 0}; fan {c, s, 0, 0}
    const float* prew;   // [nb] fan pre-weight SOD / sqrt(SOD^2 + s^2), or null
};
void launch_fbp(const FbpDev& f, int nch, const float* sino, float* q, float* x, bool clamp, cudaStream_t st);
void launch_cdm_start(int64_t n, const float* m_l, float inv_abar, float mu0, float* a_c, float* a_p, float* mu,
                      float* zero, cudaStream_t st);
void launch_unpack_meas(int64_t n, const float4* meas, float* planar, cudaStream_t st);
cudaError_t fbp_init_attributes();

// admm.cu helpers are local to that file.

// ---- error handling ----------------------------------------------------------------------
void set_error(const std::string& msg);

}  // namespace dect
