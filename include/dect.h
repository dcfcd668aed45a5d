/*
 * dect.h - C ABI of the GB300 (sm_103a) library for one ADMM iteration of the
 * splitting-based statistical dual-energy CT reconstruction UDM(m)-PCG(n)
 * (Li, Manerikar, Prakash, Kak: "A splitting-based iterative algorithm for
 * GPU-accelerated statistical dual-energy X-ray CT reconstruction").
 *
 * Conventions shared by every call
 *  - Images are row-major [ny][nx] float32; pixel (row j, column i) is centred
 *    at ((i-(nx-1)/2)*pixel_cm, (j-(ny-1)/2)*pixel_cm).
 *  - Sinograms are [n_views][n_bins] float32, bins fastest.
 *  - Multi-channel buffers are planar: channel 0 (Compton, x_c) first, then
 *    channel 1 (photoelectric, x_p), each a full image or sinogram.
 *  - "dev" pointers are device memory owned by the caller; the library never
 *    frees or keeps them past the call (asynchronous calls read/write them in
 *    stream order on the given stream). Handles own only their internal
 *    workspaces and free them in their destroy call.
 *  - stream is a cudaStream_t passed as void*; NULL means the legacy default
 *    stream. Calls on one handle must be ordered (same stream, or synchronised
 *    by the caller): a handle's workspace is shared by its calls.
 *  - Every call returns a dect_status. Arguments are validated before anything
 *    is launched; on failure nothing is launched and dect_last_error() (per
 *    host thread) describes the problem. Errors of earlier asynchronous work
 *    surface as DECT_ECUDA from a later call or from dect_sync().
 *  - No call traps or asserts on the device. Per-ray numerical failures of the
 *    decomposition are reported in a status array, not as call errors.
 */
#ifndef DECT_H
#define DECT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    DECT_OK = 0,
    DECT_EINVAL = 1,        /* bad argument (null pointer, bad size, bad enum) */
    DECT_ENOMEM = 2,        /* device or host allocation failed */
    DECT_ECUDA = 3,         /* a CUDA runtime error, from this or earlier work */
    DECT_EUNSUPPORTED = 4,  /* valid but not supported (e.g. a dtype) */
    DECT_ETIMEOUT = 5,      /* reserved: a bounded device wait ran out */
    DECT_ENOTCONV = 6       /* reserved: a solver did not converge */
} dect_status;

typedef enum { DECT_PARALLEL = 0, DECT_FAN_FLAT = 1 } dect_geom_kind;

typedef enum { DECT_F32 = 0, DECT_F64 = 1 } dect_dtype;

/* Storage format of the solver's sinogram-domain vectors (a, u^a, R x, the CG
 * sinogram) and of the projector's pair textures. With F32, F16 and BF16 the
 * arithmetic is float32 (the decomposition's by default; see
 * dect_params.udm_f64). DECT_STORE_F64 runs a separate float64 solver: every
 * vector, scalar and operation of the iteration (projector pair, FFT
 * preconditioner, decomposition, updates) in float64, for problems whose
 * photoelectric signal lies below float32 resolution (Sec. 1: the PE basis
 * decays as E^-3, so with a 1 keV reference f_p a_p is ~1e-7 of the
 * attenuation). It supports images up to 1024 x 1024, the UDM-PCG scheme and
 * the DECT_INIT_PCG start; its projector pair is a plain float64 gather
 * (much slower than the float32 kernels: meant for small problems). */
typedef enum { DECT_STORE_F32 = 0, DECT_STORE_F16 = 1, DECT_STORE_BF16 = 2, DECT_STORE_F64 = 3 } dect_storage;

/* Per-ray decomposition status codes (uint8 array of dect_decompose_rays). */
enum { DECT_RAY_ACCEPTED = 0, DECT_RAY_REJECTED = 1, DECT_RAY_NONFINITE = 2 };

/* Library version string, e.g. "dect 0.1 sm_103a". */
const char* dect_version(void);

/* Description of the last error on the calling host thread ("" if none). */
const char* dect_last_error(void);

/* Blocks until all work on `stream` is done; returns DECT_ECUDA on an asynchronous error. */
dect_status dect_sync(void* stream);

/* ------------------------------------------------------------------------ */
/* Geometry: the projection matrix R of Eq. 2-3 (Sec. 1, Sec. 3.1).
 *
 * Parallel beam (the paper's experiments, Sec. 4): view v has angle
 * theta_v = angle0_rad + v*angle_span_rad/n_views; bin k sits at
 * u_k = (k-(n_bins-1)/2)*bin_pitch_cm + bin_offset_cm; its ray passes through
 * u_k*(cos, sin)(theta_v) with direction (-sin, cos)(theta_v).
 * Fan beam, flat detector: source at sod_cm*(cos, sin)(theta_v), detector line
 * through -(sdd_cm-sod_cm)*(cos, sin)(theta_v) along (-sin, cos)(theta_v); the
 * ray of bin k runs from the source to u_k on that line.
 * R is Joseph's interpolating ray-driven projector: a ray with |d_x| >= |d_y|
 * is sampled once per image column with linear interpolation between the two
 * nearest rows (zero outside the image), weighted by pixel_cm/|d_x|; otherwise
 * rows and columns swap roles.
 * Limits: 1 <= nx, ny <= 4096; 1 <= n_views <= 16384; 1 <= n_bins <= 16384;
 * pixel_cm, bin_pitch_cm > 0; fan beam needs sdd_cm > sod_cm > 0 and the
 * image's circumscribed circle strictly inside the source circle.
 */
typedef struct {
    int32_t kind;           /* dect_geom_kind */
    int32_t nx, ny;         /* image columns, rows */
    int32_t n_views, n_bins;
    double pixel_cm;
    double angle0_rad, angle_span_rad;
    double bin_pitch_cm, bin_offset_cm;
    double sod_cm, sdd_cm;  /* fan beam only */
} dect_geom_desc;

typedef struct dect_geom dect_geom;

/* Creates a geometry on the current CUDA device (builds the per-ray table
 * there). *out receives the handle; the caller destroys it. */
dect_status dect_geometry_create(const dect_geom_desc* desc, dect_geom** out);
void dect_geometry_destroy(dect_geom* g);

/* ------------------------------------------------------------------------ */
/* Spectral tables of Eq. 1-3: f_{h/l}(a) = C_{h/l} - ln sum_E S_{h/l}(E)
 * exp(-f_KN(E) a_c - f_p(E) a_p), with the integral over E as a sum over the
 * n_energies bins. All four host arrays are FP64 of length n_energies
 * (1..512), copied during the call. S_h and S_l must be >= 0 with positive
 * sums; the library normalises them to unit sum, which makes C_{h/l} = 0. */
typedef struct dect_spectra dect_spectra;
dect_status dect_spectra_create(int32_t n_energies, const double* S_h, const double* S_l,
                                const double* f_kn, const double* f_p, dect_spectra** out);
void dect_spectra_destroy(dect_spectra* s);

/* ------------------------------------------------------------------------ */
/* Forward projection (Eq. 2-3's R): sino_dev[c] = R x_dev[c] for c < n_channels.
 * x_dev: planar [n_channels][ny][nx]; sino_dev: planar [n_channels][n_views][n_bins],
 * overwritten; both of `dtype` (DECT_F32 or DECT_F64). n_channels is 1 or 2.
 * DECT_F32 samples positions in 34.30 fixed point (~1e-7 pixel); DECT_F64 uses a
 * float64 ray table (built on first use) and float64 accumulation.
 * Uses the geometry's workspace (allocated on first use). */
dect_status dect_project(dect_geom* g, int32_t n_channels, int32_t dtype, const void* x_dev,
                         void* sino_dev, void* stream);

/* Size of the fixed scratch array used by dect_project_noalloc (4 MiB). */
#define DECT_NOALLOC_SCRATCH_BYTES (4u * 1024u * 1024u)

/* Forward projection without any device allocation. The paper has no counterpart:
 * this is a library convenience for callers that cannot call cudaMalloc (code
 * running during CUDA stream capture, code whose device memory belongs to its
 * own pool or framework allocator, fixed-budget deployments). Same operation,
 * layouts and results as dect_project, but its scratch (pair textures and an
 * interleaved image copy, 16*(nx*(ny+3) + ny*(nx+3)) + 8*nx*ny bytes) lives in
 * a fixed DECT_NOALLOC_SCRATCH_BYTES array of device global memory inside the
 * library, which every GPU that loads the library holds until exit; images up
 * to about 320 x 320 fit. Larger images are rejected with DECT_EINVAL and a
 * message, before anything is launched. The first call on a device looks up
 * the array's device address (cudaGetSymbolAddress) with that device current;
 * make that first call before any stream capture. All calls share the array:
 * calls that overlap on the GPU (other streams, other host threads) race and
 * must be ordered by the caller. Each call rewrites all scratch it reads, so
 * nothing needs clearing between calls. */
dect_status dect_project_noalloc(const dect_geom* g, int32_t n_channels, const float* x_dev, float* sino_dev,
                                 void* stream);

/* Backprojection, the exact adjoint R^T of dect_project (Table 1's R^T):
 * x_dev[c] = R^T sino_dev[c]; same layouts and dtypes; x_dev is overwritten. Every
 * pixel is accumulated by one thread (image tiles sweep the rays that reach them,
 * partial images are added in a fixed order; no atomics), so the result is
 * deterministic; it evaluates the same per-ray weights as dect_project, so
 * <R x, y> = <x, R^T y> up to float32 rounding. */
dect_status dect_backproject(dect_geom* g, int32_t n_channels, int32_t dtype, const void* sino_dev,
                             void* x_dev, void* stream);

/* ------------------------------------------------------------------------ */
/* Per-ray decomposition, Eq. 13 (UDM): for each of the n_rays rays
 *   min over (a_c, a_p) of 1/2 sum_{k=h,l} w_k (f_k(a) - m_k)^2
 *                          + rho_c/2 (a_c - v_c)^2 + rho_p/2 (a_p - v_p)^2
 * by `iters` Levenberg-Marquardt iterations from the warm start in a_c, a_p:
 * Gauss-Newton system (J^T W J + diag rho), Marquardt damping mu*diag, a step
 * is kept only if it lowers the cost (mu /= 10) else mu *= 10, mu clamped to
 * [1e-10, 1e10]; 4 evaluations of f per iteration (Table 1).
 * All arrays are device float32 of length n_rays except status (uint8,
 * nullable). a_c, a_p, mu are read and overwritten. rho = 0 gives the plain
 * maximum-likelihood decomposition. Float32 throughout: compensated sums over
 * energy, residuals as -log of the ratio of the spectral sum to the measured
 * transmission, the 2x2 Marquardt solve from the Jacobian's minors. */
dect_status dect_decompose_rays(const dect_spectra* s, int64_t n_rays, const float* m_h, const float* m_l,
                                const float* w_h, const float* w_l, const float* v_c, const float* v_p,
                                double rho_c, double rho_p, int32_t iters, float* a_c, float* a_p,
                                float* mu, uint8_t* status, void* stream);

/* ------------------------------------------------------------------------ */
/* Filtered backprojection, the reconstruction half of the CDM-FBP comparison
 * method (Sec. 2, Sec. 4): the band-limited ramp filter h(0) = 1/(4 a^2),
 * h(m a) = -1/(pi^2 m^2 a^2) for odd m, 0 for even m != 0, applied along each
 * view (linear convolution, no wrap-around), then backprojection with linear
 * interpolation between bins (zero beyond the first and last bin).
 *   parallel beam, views over pi or 2 pi (a = du): x = (pi/V) sum_v Q_v(t),
 *     t = P . (cos, sin)(theta_v);
 *   flat-detector fan beam, views over 2 pi: the detector rescaled to the
 *     isocentre (s = u SOD/SDD, a = du SOD/SDD), pre-weight SOD/sqrt(SOD^2+s^2),
 *     half the ramp, x = (2 pi/V) sum_v Q_v(s(P)) / U^2 with
 *     U = (SOD - P . n_v)/SOD, s(P) = (P . e_v)/U (n_v towards the source,
 *     e_v the detector axis, as in dect_geom_desc).
 * sino_dev: float32 [n_channels][n_views][n_bins]; x_dev: float32
 * [n_channels][ny][nx], overwritten; both device memory owned by the caller.
 * clamp_nonneg != 0 replaces negative sinogram values by 0 first (the CDM
 * constraint). n_channels is 1 or 2. Other angular spans (short scans) return
 * DECT_EUNSUPPORTED. The filtered rows live in a per-geometry workspace
 * (allocated on the first call), so calls on one geometry must be ordered. */
dect_status dect_fbp(dect_geom* g, int32_t n_channels, const float* sino_dev, float* x_dev, int32_t clamp_nonneg,
                     void* stream);

/* CDM-FBP, the comparison method of Sec. 4: per ray the decomposition of
 * dect_decompose_rays with rho_c = rho_p = 0 (the weighted least-squares fit of
 * f(a) to (m_h, m_l)) by `iters` LM iterations from a_c = m_l / sum_E S_l f_KN,
 * a_p = 0, mu = 1e-3; then a >= 0 per basis and dect_fbp of both bases.
 * m_h, m_l, w_h, w_l: float32 [n_views][n_bins] device. x_dev: float32
 * [2][ny][nx] (Compton, PE), overwritten. work_dev: NULL (the call allocates
 * and frees stream-ordered scratch) or 4 n_views n_bins floats of device memory,
 * which then hold a_c, a_p (before the clamp), mu and zeros on return. */
dect_status dect_cdm_fbp(dect_geom* g, const dect_spectra* s, const float* m_h, const float* m_l, const float* w_h,
                         const float* w_l, int32_t iters, float* work_dev, float* x_dev, void* stream);

/* Forward model of Eq. 3 per ray: f_h, f_l at (a_c, a_p) and, if jac is not
 * NULL, the Jacobian jac[r] = {df_h/da_c, df_h/da_p, df_l/da_c, df_l/da_p}
 * ([n_rays][4]). All arrays device memory of `dtype` (DECT_F32: float32
 * exponentials with compensated sums, float64 logs of the sums; DECT_F64:
 * float64 throughout). f_h, f_l may be NULL. */
dect_status dect_forward_model(const dect_spectra* s, int64_t n_rays, int32_t dtype, const void* a_c, const void* a_p,
                               void* f_h, void* f_l, void* jac, void* stream);

/* Vector-Jacobian product of the forward model (its transpose applied to an
 * output gradient): grad_c = g_h df_h/da_c + g_l df_l/da_c, grad_p likewise;
 * the backward pass of the forward model in automatic differentiation. */
dect_status dect_forward_model_vjp(const dect_spectra* s, int64_t n_rays, int32_t dtype, const void* a_c,
                                   const void* a_p, const void* g_h, const void* g_l, void* grad_c, void* grad_p,
                                   void* stream);

/* ------------------------------------------------------------------------ */
/* ADMM solver state for B >= 1 independent slices (Sec. 3.2-3.3).
 * One iteration (UDM(m)-PCG(n)), per slice and for both bases beta in {c, p}:
 *  1. Eq. 12: n preconditioned CG steps on (R^T R + D^T D + I) x_beta
 *     = R^T(a+u^a) + D^T(y+u^y) + (z+u^z), warm-started from x_beta, with
 *     R x carried (R x += alpha R p): 2n R and 2(n+1) R^T (Table 1).
 *     D: forward differences along x and y, zero at the last column/row.
 *     Preconditioner (dect_precond): the circulant model 1/(F[R^T R delta] + |F[D]|^2 + 1)
 *     of the operator on a zero-padded grid (the high-pass filter of Sec. 3.3); or the plain
 *     ramp filter 1/(K/|w| + 1) = |w|/(K + |w|), |w| the radial frequency in radians per
 *     pixel floored at the first non-zero grid frequency, K = (pi/4) F[R^T R delta](0, pi/4);
 *     or none (plain CG).
 *  2. Eq. 13: m LM iterations per ray with v = R x - u^a (as dect_decompose_rays).
 *  3. Eq. 9-10: y = shrinkage(D x - u^y, lambda/rho), z = max(0, x - u^z).
 *  4. Eq. 11 with the a-block: u^a += a - R x, u^y += y - D x, u^z += z - x.
 *  5. rho by residual balancing (Sec. 3.2): r_pri = ||[a;y;z] - [R;D;I]x||,
 *     r_dual = rho ||[a;y;z] - [a;y;z]_prev||; if r_pri > mu_b r_dual then
 *     rho *= tau, u /= tau; if r_dual > mu_b r_pri then rho /= tau, u *= tau.
 * All scalars (CG alpha/beta, rho, residuals) stay on the device.
 *
 * With scheme = DECT_SCHEME_LM_CG the iteration is instead the comparison scheme
 * LM(m) x CG(n) of Sec. 3.2 (Eq. 6-11; Table 1's first row), float32 storage only:
 *  1. Eq. 7 then Eq. 8: m Levenberg-Marquardt steps on x_c (x_p fixed), then on
 *     x_p (the new x_c fixed). A step models the data term by Gauss-Newton around
 *     the current projections and adds the basis' augmented-Lagrangian term
 *     rho/2 ||[y; z] - [D; I] x + u||^2; its linear system, with the data
 *     curvature scaled by (1 + mu), is solved by n plain CG iterations from 0;
 *     the step is kept iff the subproblem objective decreases (mu / 10), else
 *     dropped (mu * 10); one mu per slice and basis, mu0 = lm_mu0. Per step:
 *     n R and n + 1 R^T on the basis (R d is carried through CG, so the trial
 *     point needs no projection; Table 1 counts n + 1 R), 2 f-evaluations.
 *  2-4. Eq. 9-11 without an a-block; rho by residual balancing on [y; z].
 * m_udm and n_pcg give m and n. The initial image is the same as above. */
enum dect_scheme { DECT_SCHEME_UDM_PCG = 0, DECT_SCHEME_LM_CG = 1 };
enum dect_precond { DECT_PRECOND_NONE = 0, DECT_PRECOND_CIRCULANT = 1, DECT_PRECOND_RAMP = 2 };
/* Initial image when a slice has no x0 (both: x_p0 = kappa x_c0, x_c0 >= 0):
 * DECT_INIT_PCG      per-ray decomposition (init_udm_iters LM iterations, rho_c = 0, rho_p = rho0_p,
 *                    v = 0) and init_pcg_iters CG iterations on (R^T R + I) x_c = R^T a_c from 0;
 * DECT_INIT_CDM_FBP  the paper's start (Sec. 4): the Compton image of CDM-FBP (dect_cdm_fbp with
 *                    init_udm_iters LM iterations and mu0 = lm_mu0); needs full scans. */
enum dect_init { DECT_INIT_PCG = 0, DECT_INIT_CDM_FBP = 1 };

typedef struct {
    double lambda_c, lambda_p;   /* TV weights (paper: 1e-5) */
    double rho0_c, rho0_p;       /* initial penalties (paper: 1e-3) */
    int32_t m_udm, n_pcg;        /* UDM(m)-PCG(n), >= 1 */
    double rho_mu, rho_tau;      /* residual balancing (10, 2); tau = 1 disables */
    double lm_mu0;               /* initial LM damping per ray (1e-3) */
    double kappa;                /* initial PE image = kappa * Compton image */
    int32_t init_udm_iters;      /* initialisation: LM iterations (10) */
    int32_t init_pcg_iters;      /* initialisation: CG iterations (10) */
    int32_t precondition;        /* enum dect_precond: 1 circulant model (default), 2 ramp filter,
                                    0 plain CG; other values: DECT_EINVAL */
    int32_t use_graph;           /* 1: capture one iteration as a CUDA graph */
    int32_t bp_view_groups;      /* backprojector view groups per image tile, 1..16; -1 = chosen from the
                                    occupancy (fill the GPU's resident slots) without timing; 0 = autotuned:
                                    dect_admm_create times the backprojector on this batch for a few
                                    candidates (memory permitting) and keeps the fastest (reported in
                                    dect_stats). It fixes the order of a pixel's partial sums: results
                                    are bitwise reproducible for a fixed value, and a slice solved alone
                                    or in a batch gives identical bits when the value is the same (it is
                                    the one launch-dependent choice; an autotuned value can differ from
                                    run to run). */
    int32_t storage;             /* dect_storage (DECT_STORE_F32): 16-bit formats halve the bytes of the
                                    sinogram vectors and textures at the cost of their precision */
    int32_t scheme;              /* dect_scheme (DECT_SCHEME_UDM_PCG): the splitting one iteration runs */
    int32_t init;                /* dect_init (DECT_INIT_PCG): the initial image of slices without x0 */
    int32_t udm_f64;             /* float32 / float16 / bfloat16 storage only. 0 (default): the decomposition
                                    (Eq. 13) in float32 as described at dect_decompose_rays. 1: float64 where
                                    the photoelectric coordinate needs it (Sec. 1): the energy sums of the
                                    spectral model accumulate the float32 exponentials in float64, its logs,
                                    the 2x2 Marquardt solve and the accept test (cost comparison) are float64.
                                    Float64 runs at 1/64 of the float32 rate on this GPU, so this is several
                                    times slower than 0 (the cost per slice is reported by the bench). */
    int32_t objective_every;     /* k > 0: after every k-th iteration (counted from the last dect_reconstruct
                                    or initialisation) the solver evaluates the MAP objective of Eq. 4 at the
                                    current images, 1/2 ||f(R x) - m||^2_Sigma + sum_b lambda_b ||D x_b||_1
                                    (R x projected afresh, f and the residuals as in the decomposition; with
                                    16-bit storage R x carries the storage's rounding), reported by
                                    dect_admm_stats. One projection and one f-evaluation per ray each time,
                                    outside Table 1's counts. 0 (default): never. */
    int32_t bp_tile;             /* backprojector tile side in pixels, 32 or 64 (its CTA's warps take bands of
                                    32 columns or rows of the tile); 0 (default) = chosen by the autotuner
                                    with bp_view_groups (timed on this batch; with bp_view_groups fixed, the
                                    two sides are timed at that count; with -1, 32). The side does not change
                                    results (every pixel receives the same contributions in the same order). */
    int32_t bp_cluster;          /* the backprojector's view groups of a tile as one thread-block cluster that
                                    adds their accumulators on chip (distributed shared memory, in rank order)
                                    into one partial image, instead of C partial images through L2 / DRAM:
                                    1 on (2 <= view groups <= 16; one slice per CTA, so bp_slices = 2 with
                                    it is DECT_EINVAL), -1 off, 0 (default) timed by the autotuner against
                                    the plain form. Both forms give the same bits. */
    int32_t bp_slices;           /* slices per backprojector CTA: 2 backprojects the same rays into two
                                    consecutive slices of one geometry at once (shared staging and sample
                                    positions, one accumulator per slice; UDM-PCG scheme), 1 one slice,
                                    0 (default) timed by the autotuner (one slice when bp_cluster = 1).
                                    Same bits either way. */
    int32_t bp_reduce;           /* plain (non-cluster) backprojector with C >= 2 view groups: the last CTA of a
                                    tile to finish sums the tile's C partial images (in view-group order, the
                                    finalize pass's order) into partial image 0 while they are in L2 and drops
                                    the other partials' L2 lines, so they are not written back to DRAM; the
                                    finalize pass reads one image. 0 (default) or 1 on, -1 off (the finalize
                                    pass reads the C partials). Same bits either way. */
    int32_t proj_views;          /* views per forward-projector CTA (tiles of views x 32 bins): 2, 4 or 8, or 0
                                    (default) timed at creation. Same bits either way. */
} dect_params;

/* Fills *p with the paper's values and the defaults above. */
void dect_params_default(dect_params* p);

typedef struct dect_admm dect_admm;

/* Creates the solver for B slices; geoms[b] describes slice b (the handles must
 * outlive the solver). Allocates all state on the current device and computes
 * each slice's preconditioner. */
dect_status dect_admm_create(dect_geom* const* geoms, int32_t n_slices, const dect_spectra* s,
                             const dect_params* p, dect_admm** out);
void dect_admm_destroy(dect_admm* a);

/* Measurements of slice b: m_h, m_l (log projections, Eq. 2) and w_h, w_l (the
 * photon counts on the diagonal of Sigma, Eq. 4), each [n_views][n_bins]
 * float32, in host or device memory (copied in stream order). If x0 is
 * non-NULL it is the starting image, planar [2][ny][nx] float32 (host or
 * device); otherwise the next dect_reconstruct computes one (see there). */
dect_status dect_admm_set_data(dect_admm* a, int32_t slice, const float* m_h, const float* m_l,
                               const float* w_h, const float* w_l, const float* x0, void* stream);

/* Ground truth [2][ny][nx] float32 (host or device) for the quality metric
 * xi (Eq. 14) of slice b; NULL clears it. */
dect_status dect_admm_set_truth(dect_admm* a, int32_t slice, const float* truth, void* stream);

/* Runs `iters` ADMM iterations on all slices. */
dect_status dect_admm_step(dect_admm* a, int32_t iters, void* stream);

/* Starts every slice that has no starting image from the initial estimate:
 * a = Eq. 13 with rho = (0, rho0_p), v = 0, from a_c = m_l / sum_E S_l f_KN,
 * a_p = 0 (init_udm_iters LM iterations); x_c = max(0, init_pcg_iters CG
 * iterations on (R^T R + I) x = R^T a_c from 0); x_p = kappa x_c. Then every
 * slice is reset to x, R x, a = R x, y = D x, z = x, zero duals, rho = rho0,
 * mu = lm_mu0; then runs `iters` iterations. */
dect_status dect_reconstruct(dect_admm* a, int32_t iters, void* stream);

/* Copies a state array of slice b to dst (host or device), planar float32
 * (float64 with DECT_STORE_F64 storage, except which = 8 and 9, which are float64 there too):
 * which = 0: x [2][ny][nx]; 1: R x [2][V][Nb]; 2: a [2][V][Nb]; 3: u^a;
 * 4: y [2][2][ny][nx] (channel, then component along x, along y); 5: u^y;
 * 6: z [2][ny][nx]; 7: u^z; 8: LM mu [V][Nb]; 9: the preconditioner
 * response H [Py][Px] (float32). dst_bytes is checked against the size. */
dect_status dect_admm_get(const dect_admm* a, int32_t slice, int32_t which, void* dst, size_t dst_bytes,
                          void* stream);

/* Per-slice scalars after the last completed iteration (synchronises `stream`). */
typedef struct {
    int32_t iteration;
    double rho[2];
    double r_pri[2], r_dual[2];
    double xi_db[2];             /* Eq. 14 against the truth (NaN without one) */
    int64_t count_R, count_RT;   /* projector applications per basis (Table 1) */
    int64_t count_f;             /* forward-model evaluations per ray */
    int64_t count_launches;      /* kernels launched by this solver so far (all slices) */
    int32_t bp_view_groups;      /* backprojector view groups per tile in use (fixed or autotuned) */
    double objective;            /* Eq. 4 after iteration objective_iteration (NaN if never evaluated) */
    int32_t objective_iteration; /* see dect_params.objective_every; -1 if never evaluated */
    int32_t bp_tile;             /* backprojector tile side in use (0 for float64 storage) */
    int32_t bp_cluster;          /* 1 if the backprojector's view groups reduce on chip (see bp_cluster) */
    int32_t bp_slices;           /* slices per backprojector CTA in use (see bp_slices; 0 for float64) */
    int32_t bp_reduce;           /* 1 if the backprojector's view groups are summed by its last CTA per tile */
    int32_t proj_views;          /* views per forward-projector CTA in use (0 for float64 storage) */
} dect_stats;
dect_status dect_admm_stats(dect_admm* a, int32_t slice, dect_stats* out, void* stream);

/* Checkpoint and resume of a solver. The state image holds, for every slice, the
 * iterate of Sec. 3.2-3.3 (x, R x, a, y, z and the scaled duals u^a, u^y, u^z),
 * rho and the per-slice scalars, the LM damping and status per ray, the CG
 * vectors, the comparison scheme's vectors and scalars, the measurements, x0 and
 * the truth, and the host-side counters; not the geometry, spectra or
 * parameters, nor what is derived from them (textures, preconditioner).
 * dect_admm_state_bytes: the image's size in bytes.
 * dect_admm_save: writes the image to host memory dst_host (capacity `bytes`,
 * at least the size; caller-owned) after the work already queued on `stream`,
 * and synchronises `stream`.
 * dect_admm_load: restores an image into a solver created with the same slice
 * shapes (nx, ny, n_views, n_bins per slice, in order), storage, scheme and
 * iteration parameters (lambda, rho0, m, n, residual balancing, LM damping,
 * kappa, the start's iteration counts, preconditioner, start, udm_f64 and the
 * backprojector view groups in use); anything else, or a wrong size or header,
 * returns DECT_EINVAL without touching the solver's state. With the same parameters, dect_admm_step then
 * continues exactly (bit for bit) as the saved solver would have. Synchronises
 * `stream`. */
dect_status dect_admm_state_bytes(const dect_admm* a, size_t* bytes);
dect_status dect_admm_save(dect_admm* a, void* dst_host, size_t bytes, void* stream);
dect_status dect_admm_load(dect_admm* a, const void* src_host, size_t bytes, void* stream);

/* Kernel groups timed by dect_admm_profile. */
enum {
    DECT_PHASE_TEXTURE = 0,      /* pair textures of the image the projector reads */
    DECT_PHASE_PROJECT = 1,      /* R */
    DECT_PHASE_BACKPROJECT = 2,  /* R^T: the tile sweep writing partial images */
    DECT_PHASE_PRECOND = 3,      /* FFT preconditioner (3 kernels) */
    DECT_PHASE_UDM = 4,          /* Eq. 13 with the a-block dual update */
    DECT_PHASE_UPDATE = 5,       /* element-wise CG, Eq. 9-11 and dual rescaling kernels */
    DECT_PHASE_REDUCE = 6,       /* per-slice scalar reductions (CG alpha/beta, rho) */
    DECT_PHASE_BP_FINALIZE = 7,  /* R^T: sum of the partial images and the CG epilogues of Eq. 12 */
    DECT_NUM_PHASES = 8
};

/* Runs `iters` iterations exactly like dect_admm_step (same kernels, replayed as a
 * CUDA graph) but with a CUDA event before and after every kernel group, and
 * synchronises `stream` after each iteration to read them: adds each group's
 * device time (ms) to ms[phase] and its kernel launches to launches[phase]
 * (both arrays of DECT_NUM_PHASES, caller-owned host memory, not cleared). */
dect_status dect_admm_profile(dect_admm* a, int32_t iters, void* stream, double* ms, int64_t* launches);

#ifdef __cplusplus
}
#endif

#endif /* DECT_H */
