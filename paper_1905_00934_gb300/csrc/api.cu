// C ABI of the dect library (include/dect.h): handles, argument validation and
// the host-side orchestration of one ADMM iteration of UDM(m)-PCG(n)
// (Sec. 3.3 of the paper). Every step of the iteration runs in this library's
// kernels; the host only enqueues them (or replays them as one CUDA graph).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "admm_kernels.cuh"
#include "dect_internal.cuh"
#include "prec.cuh"

namespace dect {
static thread_local std::string g_err;
void set_error(const std::string& m) { g_err = m; }

void project_single(const SliceDesc& sd, const float* img, int nch, float2* scratch, float4* tx, float4* ty,
                    float* out, cudaStream_t st);
void launch_identity_precond(const SliceDesc* d, const BlockMap& rows, int nrows, const float2* r, float2* s,
                             double* partial, cudaStream_t st);
}  // namespace dect

using namespace dect;

#define DECT_FAIL(code, msg)   \
    do {                       \
        dect::set_error(msg);  \
        return code;           \
    } while (0)

#define CUDA_TRY(call)                                                                       \
    do {                                                                                     \
        cudaError_t e_ = (call);                                                             \
        if (e_ != cudaSuccess) {                                                             \
            dect::set_error(std::string(#call) + ": " + cudaGetErrorString(e_));             \
            return e_ == cudaErrorMemoryAllocation ? DECT_ENOMEM : DECT_ECUDA;               \
        }                                                                                    \
    } while (0)

static cudaStream_t as_stream(void* s) { return reinterpret_cast<cudaStream_t>(s); }

template <typename T>
static cudaError_t dalloc(T** p, size_t count) {
    *p = nullptr;
    if (count == 0) count = 1;
    return cudaMalloc((void**)p, count * sizeof(T));
}

static int ilog2(int v) {
    int l = 0;
    while ((1 << l) < v) ++l;
    return l;
}

static int pad_pow2(int n) {
    int p = 1;
    while (p < 2 * n) p *= 2;
    return p;
}

// ----------------------------------------------------------------------------------------------
struct dect_geom {
    dect_geom_desc desc{};
    int4* rays = nullptr;
    float4* views = nullptr;
    // workspace of dect_project / dect_backproject (allocated on first use)
    float2* ws_img = nullptr;
    float4* ws_tx = nullptr;
    float4* ws_ty = nullptr;
    float2* ws_sino = nullptr;
    // R^T workspace: descriptor with zero offsets, block-map prefixes {0, sweep CTAs, 0, pixel blocks},
    // ws_C partial images
    SliceDesc* ws_desc = nullptr;
    int* ws_maps = nullptr;
    float2* ws_partial = nullptr;
    int ws_C = 1;
    double4_32a* rays64 = nullptr;  // float64 ray table (DECT_F64 calls; built on first use)
    // dect_fbp: per-view constants, fan pre-weights, filtered sinograms [2][V][Nb] (built on first use)
    float4* fbp_tab = nullptr;
    float* fbp_prew = nullptr;
    float* fbp_q = nullptr;

    int64_t n_rays() const { return (int64_t)desc.n_views * desc.n_bins; }
    int64_t n_pix() const { return (int64_t)desc.nx * desc.ny; }
    GeomDev dev() const {
        GeomDev g;
        g.kind = desc.kind;
        g.nx = desc.nx;
        g.ny = desc.ny;
        g.nv = desc.n_views;
        g.nb = desc.n_bins;
        g.pix = (float)desc.pixel_cm;
        g.du = (float)desc.bin_pitch_cm;
        g.uoff = (float)desc.bin_offset_cm;
        g.sod = (float)desc.sod_cm;
        g.sdd = (float)desc.sdd_cm;
        g.cx = 0.5f * (float)(desc.nx - 1);
        g.cy = 0.5f * (float)(desc.ny - 1);
        g.inv_du = (float)(1.0 / desc.bin_pitch_cm);
        g.k0 = (float)(0.5 * (desc.n_bins - 1) - desc.bin_offset_cm / desc.bin_pitch_cm);
        g.k1 = (float)(desc.sdd_cm / desc.bin_pitch_cm);
        g.rays = rays;
        g.views = views;
        return g;
    }
    SliceDesc single() const {
        SliceDesc s{};
        s.g = dev();
        return s;
    }
};

namespace dect {
// accessors for the no-allocation projector (project_noalloc.cu)
const dect_geom_desc* geom_desc_of(const dect_geom* g) { return &g->desc; }
SliceDesc geom_single_of(const dect_geom* g) { return g->single(); }
}  // namespace dect

struct dect_spectra {
    int ne = 0;
    float4* t1 = nullptr;
    float4* t2 = nullptr;
    double4_32a* t64 = nullptr;  // {S_h, S_l, f_KN, f_p}, unit-sum spectra
    double4_32a* w64 = nullptr;  // [2][ne]: {S_h, S_l, S_h f_KN, S_h f_p}, {S_l f_KN, S_l f_p, 0, 0}
    double abar_low = 1.0;  // sum_E S_l f_KN (unit-sum S_l)
    int n_both = 0, n_end = 0, tail_high = 1;  // supports of the spectra (see SpecDev)
    SpecDev dev() const { return SpecDev{ne, t1, t2, w64, w64 + ne, n_both, n_end, tail_high}; }
};

extern "C" const char* dect_version(void) { return "dect 0.1 sm_103a"; }
extern "C" const char* dect_last_error(void) { return dect::g_err.c_str(); }

extern "C" dect_status dect_sync(void* stream) {
    CUDA_TRY(cudaStreamSynchronize(as_stream(stream)));
    CUDA_TRY(cudaGetLastError());
    return DECT_OK;
}

static bool finite_pos(double v) { return std::isfinite(v) && v > 0.0; }

static bool same_geometry(const dect_geom_desc& a, const dect_geom_desc& b) {
    return a.kind == b.kind && a.nx == b.nx && a.ny == b.ny && a.n_views == b.n_views && a.n_bins == b.n_bins &&
           a.pixel_cm == b.pixel_cm && a.angle0_rad == b.angle0_rad && a.angle_span_rad == b.angle_span_rad &&
           a.bin_pitch_cm == b.bin_pitch_cm && a.bin_offset_cm == b.bin_offset_cm && a.sod_cm == b.sod_cm &&
           a.sdd_cm == b.sdd_cm;
}

// Launch errors are read back with cudaGetLastError; clear any error left by an unrelated earlier
// runtime call so that it is not reported against this call.
static void clear_stale_error() { (void)cudaGetLastError(); }

extern "C" dect_status dect_geometry_create(const dect_geom_desc* d, dect_geom** out) {
    clear_stale_error();
    if (!d || !out) DECT_FAIL(DECT_EINVAL, "dect_geometry_create: null argument");
    *out = nullptr;
    if (d->kind != DECT_PARALLEL && d->kind != DECT_FAN_FLAT) DECT_FAIL(DECT_EINVAL, "geometry: unknown kind");
    if (d->nx < 1 || d->ny < 1 || d->nx > 4096 || d->ny > 4096) DECT_FAIL(DECT_EINVAL, "geometry: nx, ny must be in [1, 4096]");
    if (d->n_views < 1 || d->n_bins < 1 || d->n_views > 16384 || d->n_bins > 16384)
        DECT_FAIL(DECT_EINVAL, "geometry: n_views, n_bins must be in [1, 16384]");
    if (!finite_pos(d->pixel_cm) || !finite_pos(d->bin_pitch_cm)) DECT_FAIL(DECT_EINVAL, "geometry: pixel and bin pitch must be > 0");
    if (!std::isfinite(d->angle0_rad) || !std::isfinite(d->angle_span_rad) || !std::isfinite(d->bin_offset_cm))
        DECT_FAIL(DECT_EINVAL, "geometry: non-finite angle or offset");
    if (d->kind == DECT_FAN_FLAT) {
        if (!finite_pos(d->sod_cm) || !finite_pos(d->sdd_cm) || d->sdd_cm <= d->sod_cm)
            DECT_FAIL(DECT_EINVAL, "geometry: fan beam needs sdd > sod > 0");
        const double r = 0.5 * d->pixel_cm * std::sqrt((double)d->nx * d->nx + (double)d->ny * d->ny) + 2.0 * d->pixel_cm;
        if (r >= 0.98 * d->sod_cm) DECT_FAIL(DECT_EINVAL, "geometry: image must lie well inside the source circle");
        // the backprojectors project rectangles around image tiles onto the detector, which needs
        // them in front of the source with a margin
        if (d->sod_cm - r < 4.25 * d->pixel_cm) DECT_FAIL(DECT_EINVAL, "geometry: source too close to the image");
    }
    dect_geom* g = new dect_geom();
    g->desc = *d;
    cudaError_t e = dalloc(&g->rays, (size_t)g->n_rays());
    if (e == cudaSuccess) e = dalloc(&g->views, (size_t)d->n_views);
    if (e == cudaSuccess) e = build_ray_table(*d, g->rays, g->views, 0);
    if (e == cudaSuccess) e = cudaStreamSynchronize(0);
    if (e != cudaSuccess) {
        dect::set_error(std::string("dect_geometry_create: ") + cudaGetErrorString(e));
        dect_geometry_destroy(g);
        return e == cudaErrorMemoryAllocation ? DECT_ENOMEM : DECT_ECUDA;
    }
    *out = g;
    return DECT_OK;
}

extern "C" void dect_geometry_destroy(dect_geom* g) {
    if (!g) return;
    cudaFree(g->rays);
    cudaFree(g->views);
    cudaFree(g->ws_img);
    cudaFree(g->ws_tx);
    cudaFree(g->ws_ty);
    cudaFree(g->ws_sino);
    cudaFree(g->ws_desc);
    cudaFree(g->ws_maps);
    cudaFree(g->ws_partial);
    cudaFree(g->rays64);
    cudaFree(g->fbp_tab);
    cudaFree(g->fbp_prew);
    cudaFree(g->fbp_q);
    delete g;
}

static dect_status geom_workspace(dect_geom* g) {
    if (g->ws_img) return DECT_OK;
    const auto& d = g->desc;
    CUDA_TRY(dalloc(&g->ws_img, (size_t)g->n_pix()));
    CUDA_TRY(dalloc(&g->ws_tx, (size_t)d.nx * (d.ny + 3)));
    CUDA_TRY(dalloc(&g->ws_ty, (size_t)d.ny * (d.nx + 3)));
    CUDA_TRY(dalloc(&g->ws_sino, (size_t)g->n_rays()));
    CUDA_TRY(sweep_init_attributes());  // per device: the geometry's device is the current one
    const int tiles = sweep_tiles(d.nx, d.ny, kSweepTileDefault);
    g->ws_C = sweep_groups(tiles, kSweepTileDefault);
    CUDA_TRY(dalloc(&g->ws_partial, (size_t)g->ws_C * g->n_pix()));
    CUDA_TRY(dalloc(&g->ws_desc, 1));
    CUDA_TRY(dalloc(&g->ws_maps, 4));
    const SliceDesc sd = g->single();
    const int maps[4] = {0, tiles * g->ws_C, 0, (int)((g->n_pix() + kPixPerBlock - 1) / kPixPerBlock)};
    CUDA_TRY(cudaMemcpy(g->ws_desc, &sd, sizeof(SliceDesc), cudaMemcpyHostToDevice));
    CUDA_TRY(cudaMemcpy(g->ws_maps, maps, sizeof(maps), cudaMemcpyHostToDevice));
    return DECT_OK;
}

static dect_status geom_table_f64(dect_geom* g) {
    if (g->rays64) return DECT_OK;
    CUDA_TRY(dalloc(&g->rays64, (size_t)g->n_rays()));
    CUDA_TRY(build_ray_table_f64(g->desc, g->rays64, 0));
    CUDA_TRY(cudaStreamSynchronize(0));
    return DECT_OK;
}

extern "C" dect_status dect_project(dect_geom* g, int32_t nch, int32_t dtype, const void* x, void* sino, void* stream) {
    clear_stale_error();
    if (!g || !x || !sino) DECT_FAIL(DECT_EINVAL, "dect_project: null argument");
    if (nch != 1 && nch != 2) DECT_FAIL(DECT_EINVAL, "dect_project: n_channels must be 1 or 2");
    if (dtype != DECT_F32 && dtype != DECT_F64) DECT_FAIL(DECT_EUNSUPPORTED, "dect_project: dtype must be DECT_F32 or DECT_F64");
    if (dtype == DECT_F64) {
        dect_status s64 = geom_table_f64(g);
        if (s64 != DECT_OK) return s64;
        project_single_f64(g->dev(), g->rays64, (const double*)x, nch, (double*)sino, as_stream(stream));
        CUDA_TRY(cudaGetLastError());
        return DECT_OK;
    }
    dect_status st = geom_workspace(g);
    if (st != DECT_OK) return st;
    project_single(g->single(), (const float*)x, nch, g->ws_img, g->ws_tx, g->ws_ty, (float*)sino, as_stream(stream));
    CUDA_TRY(cudaGetLastError());
    return DECT_OK;
}

extern "C" dect_status dect_backproject(dect_geom* g, int32_t nch, int32_t dtype, const void* sino, void* x,
                                        void* stream) {
    clear_stale_error();
    if (!g || !x || !sino) DECT_FAIL(DECT_EINVAL, "dect_backproject: null argument");
    if (nch != 1 && nch != 2) DECT_FAIL(DECT_EINVAL, "dect_backproject: n_channels must be 1 or 2");
    if (dtype != DECT_F32 && dtype != DECT_F64)
        DECT_FAIL(DECT_EUNSUPPORTED, "dect_backproject: dtype must be DECT_F32 or DECT_F64");
    if (dtype == DECT_F64) {
        dect_status s64 = geom_table_f64(g);
        if (s64 != DECT_OK) return s64;
        backproject_single_f64(g->dev(), g->rays64, (const double*)sino, nch, (double*)x, as_stream(stream));
        CUDA_TRY(cudaGetLastError());
        return DECT_OK;
    }
    dect_status st = geom_workspace(g);
    if (st != DECT_OK) return st;
    backproject_single(g->single(), g->ws_desc, g->ws_maps, g->ws_C, kSweepTileDefault, (const float*)sino, nch,
                       g->ws_sino, g->ws_partial, (float*)x, as_stream(stream));
    CUDA_TRY(cudaGetLastError());
    return DECT_OK;
}

// ----------------------------------------------------------------------------------------------
extern "C" dect_status dect_spectra_create(int32_t ne, const double* S_h, const double* S_l, const double* f_kn,
                                           const double* f_p, dect_spectra** out) {
    clear_stale_error();
    if (!out || !S_h || !S_l || !f_kn || !f_p) DECT_FAIL(DECT_EINVAL, "dect_spectra_create: null argument");
    *out = nullptr;
    if (ne < 1 || ne > kMaxEnergies) DECT_FAIL(DECT_EINVAL, "dect_spectra_create: n_energies must be in [1, 512]");
    double th = 0.0, tl = 0.0;
    for (int e = 0; e < ne; ++e) {
        if (!(S_h[e] >= 0.0) || !(S_l[e] >= 0.0) || !std::isfinite(S_h[e]) || !std::isfinite(S_l[e]) ||
            !std::isfinite(f_kn[e]) || !std::isfinite(f_p[e]))
            DECT_FAIL(DECT_EINVAL, "dect_spectra_create: spectra must be finite and >= 0, basis functions finite");
        th += S_h[e];
        tl += S_l[e];
    }
    if (!(th > 0.0) || !(tl > 0.0)) DECT_FAIL(DECT_EINVAL, "dect_spectra_create: spectra must have positive sums");
    const double log2e = 1.4426950408889634;
    std::vector<float4> t1(ne), t2(ne);
    std::vector<double4_32a> t64(ne), w64(2 * (size_t)ne);
    double abar = 0.0;
    for (int e = 0; e < ne; ++e) {
        const double sh = S_h[e] / th, sl = S_l[e] / tl;
        t64[e] = make_double4_32a(sh, sl, f_kn[e], f_p[e]);
        w64[e] = make_double4_32a(sh, sl, sh * f_kn[e], sh * f_p[e]);
        w64[ne + e] = make_double4_32a(sl * f_kn[e], sl * f_p[e], 0.0, 0.0);
        t1[e] = make_float4((float)(f_kn[e] * log2e), (float)(f_p[e] * log2e), (float)sh, (float)sl);
        t2[e] = make_float4((float)(sh * f_kn[e]), (float)(sh * f_p[e]), (float)(sl * f_kn[e]), (float)(sl * f_p[e]));
        abar += sl * f_kn[e];
    }
    dect_spectra* s = new dect_spectra();
    s->ne = ne;
    s->abar_low = abar;
    int last_h = 0, last_l = 0;  // one past the last non-zero bin of each spectrum
    for (int e = 0; e < ne; ++e) {
        if (S_h[e] > 0.0) last_h = e + 1;
        if (S_l[e] > 0.0) last_l = e + 1;
    }
    s->n_both = std::min(last_h, last_l);
    s->n_end = std::max(last_h, last_l);
    s->tail_high = last_h >= last_l ? 1 : 0;
    cudaError_t e = dalloc(&s->t1, ne);
    if (e == cudaSuccess) e = dalloc(&s->t2, ne);
    if (e == cudaSuccess) e = cudaMemcpy(s->t1, t1.data(), sizeof(float4) * ne, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(s->t2, t2.data(), sizeof(float4) * ne, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = dalloc(&s->t64, ne);
    if (e == cudaSuccess) e = cudaMemcpy(s->t64, t64.data(), sizeof(double4_32a) * ne, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = dalloc(&s->w64, 2 * (size_t)ne);
    if (e == cudaSuccess) e = cudaMemcpy(s->w64, w64.data(), sizeof(double4_32a) * 2 * ne, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        dect::set_error(std::string("dect_spectra_create: ") + cudaGetErrorString(e));
        dect_spectra_destroy(s);
        return DECT_ECUDA;
    }
    *out = s;
    return DECT_OK;
}

extern "C" void dect_spectra_destroy(dect_spectra* s) {
    if (!s) return;
    cudaFree(s->t1);
    cudaFree(s->t2);
    cudaFree(s->t64);
    cudaFree(s->w64);
    delete s;
}

extern "C" dect_status dect_decompose_rays(const dect_spectra* s, int64_t n, const float* m_h, const float* m_l,
                                           const float* w_h, const float* w_l, const float* v_c, const float* v_p,
                                           double rho_c, double rho_p, int32_t iters, float* a_c, float* a_p,
                                           float* mu, uint8_t* status, void* stream) {
    clear_stale_error();
    if (!s) DECT_FAIL(DECT_EINVAL, "dect_decompose_rays: null spectra");
    if (n < 0) DECT_FAIL(DECT_EINVAL, "dect_decompose_rays: n_rays < 0");
    if (n == 0) return DECT_OK;
    if (!m_h || !m_l || !w_h || !w_l || !v_c || !v_p || !a_c || !a_p || !mu)
        DECT_FAIL(DECT_EINVAL, "dect_decompose_rays: null array");
    if (iters < 0) DECT_FAIL(DECT_EINVAL, "dect_decompose_rays: iters < 0");
    if (!(rho_c >= 0.0) || !(rho_p >= 0.0) || !std::isfinite(rho_c) || !std::isfinite(rho_p))
        DECT_FAIL(DECT_EINVAL, "dect_decompose_rays: rho must be finite and >= 0");
    launch_udm_rays(s->dev(), n, m_h, m_l, w_h, w_l, v_c, v_p, rho_c, rho_p, iters, a_c, a_p, mu, status,
                    as_stream(stream));
    CUDA_TRY(cudaGetLastError());
    return DECT_OK;
}

// ---- FBP and CDM-FBP ---------------------------------------------------------------------------

static bool span_is(double span, double target) { return std::fabs(span - target) <= 1e-6 * target; }

static dect_status fbp_prepare(dect_geom* g, FbpDev& f) {
    const auto& d = g->desc;
    const bool fan = d.kind == DECT_FAN_FLAT;
    if (fan ? !span_is(d.angle_span_rad, 2.0 * M_PI)
            : !(span_is(d.angle_span_rad, M_PI) || span_is(d.angle_span_rad, 2.0 * M_PI)))
        DECT_FAIL(DECT_EUNSUPPORTED, "dect_fbp: views must cover 2 pi (fan) or pi / 2 pi (parallel); short scans "
                                     "are not supported");
    const double k0 = 0.5 * (d.n_bins - 1) - d.bin_offset_cm / d.bin_pitch_cm;
    if (!g->fbp_tab) {
        CUDA_TRY(fbp_init_attributes());  // per device: the geometry's device is the current one
        std::vector<float4> tab(d.n_views);
        for (int v = 0; v < d.n_views; ++v) {
            const double th = d.angle0_rad + v * (d.angle_span_rad / d.n_views);
            const double c = std::cos(th), sn = std::sin(th);
            tab[v] = fan ? make_float4((float)c, (float)sn, 0.f, 0.f)
                         : make_float4((float)(c / d.bin_pitch_cm), (float)(sn / d.bin_pitch_cm), (float)k0, 0.f);
        }
        float4* dt = nullptr;
        CUDA_TRY(dalloc(&dt, tab.size()));
        cudaError_t e = cudaMemcpy(dt, tab.data(), sizeof(float4) * tab.size(), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) {
            cudaFree(dt);
            CUDA_TRY(e);
        }
        float* pw = nullptr;
        if (fan) {
            std::vector<float> w(d.n_bins);
            for (int k = 0; k < d.n_bins; ++k) {
                const double u = (k - 0.5 * (d.n_bins - 1)) * d.bin_pitch_cm + d.bin_offset_cm;
                const double s = u * d.sod_cm / d.sdd_cm;
                w[k] = (float)(d.sod_cm / std::sqrt(d.sod_cm * d.sod_cm + s * s));
            }
            e = dalloc(&pw, w.size());
            if (e == cudaSuccess) e = cudaMemcpy(pw, w.data(), sizeof(float) * w.size(), cudaMemcpyHostToDevice);
        }
        float* q = nullptr;
        if (e == cudaSuccess) e = dalloc(&q, (size_t)2 * g->n_rays());
        if (e != cudaSuccess) {
            cudaFree(dt);
            cudaFree(pw);
            cudaFree(q);
            CUDA_TRY(e);
        }
        g->fbp_tab = dt;
        g->fbp_prew = pw;
        g->fbp_q = q;
    }
    f.nx = d.nx;
    f.ny = d.ny;
    f.nv = d.n_views;
    f.nb = d.n_bins;
    f.fan = fan ? 1 : 0;
    f.pix = (float)d.pixel_cm;
    f.cx = 0.5f * (float)(d.nx - 1);
    f.cy = 0.5f * (float)(d.ny - 1);
    f.sod = (float)d.sod_cm;
    f.k0 = (float)k0;
    f.k1 = fan ? (float)(d.sdd_cm / d.bin_pitch_cm) : 0.f;
    f.gain = fan ? (float)(0.5 * d.sdd_cm / (d.bin_pitch_cm * d.sod_cm)) : (float)(1.0 / d.bin_pitch_cm);
    f.scale = (float)((fan ? 2.0 * M_PI : M_PI) / d.n_views);
    f.tab = g->fbp_tab;
    f.prew = g->fbp_prew;
    return DECT_OK;
}

extern "C" dect_status dect_fbp(dect_geom* g, int32_t n_channels, const float* sino_dev, float* x_dev,
                                int32_t clamp_nonneg, void* stream) {
    clear_stale_error();
    if (!g || !sino_dev || !x_dev) DECT_FAIL(DECT_EINVAL, "dect_fbp: null argument");
    if (n_channels != 1 && n_channels != 2) DECT_FAIL(DECT_EINVAL, "dect_fbp: n_channels must be 1 or 2");
    FbpDev f{};
    const dect_status s = fbp_prepare(g, f);
    if (s != DECT_OK) return s;
    launch_fbp(f, n_channels, sino_dev, g->fbp_q, x_dev, clamp_nonneg != 0, as_stream(stream));
    CUDA_TRY(cudaGetLastError());
    return DECT_OK;
}

extern "C" dect_status dect_cdm_fbp(dect_geom* g, const dect_spectra* sp, const float* m_h, const float* m_l,
                                    const float* w_h, const float* w_l, int32_t iters, float* work_dev, float* x_dev,
                                    void* stream) {
    clear_stale_error();
    if (!g || !sp || !m_h || !m_l || !w_h || !w_l || !x_dev) DECT_FAIL(DECT_EINVAL, "dect_cdm_fbp: null argument");
    if (iters < 0) DECT_FAIL(DECT_EINVAL, "dect_cdm_fbp: iters < 0");
    FbpDev f{};
    const dect_status s = fbp_prepare(g, f);
    if (s != DECT_OK) return s;
    cudaStream_t st = as_stream(stream);
    const int64_t n = g->n_rays();
    float* w = work_dev;
    if (!w) CUDA_TRY(cudaMallocAsync((void**)&w, sizeof(float) * 4 * (size_t)n, st));
    float *a_c = w, *a_p = w + n, *mu = w + 2 * n, *zero = w + 3 * n;
    launch_cdm_start(n, m_l, (float)(1.0 / sp->abar_low), 1e-3f, a_c, a_p, mu, zero, st);
    launch_udm_rays(sp->dev(), n, m_h, m_l, w_h, w_l, zero, zero, 0.0, 0.0, iters, a_c, a_p, mu, nullptr, st);
    launch_fbp(f, 2, a_c, g->fbp_q, x_dev, true, st);
    cudaError_t e = cudaGetLastError();
    if (!work_dev) {
        cudaError_t fe = cudaFreeAsync(w, st);
        if (e == cudaSuccess) e = fe;
    }
    CUDA_TRY(e);
    return DECT_OK;
}

extern "C" dect_status dect_forward_model(const dect_spectra* s, int64_t n, int32_t dtype, const void* a_c,
                                          const void* a_p, void* f_h, void* f_l, void* jac, void* stream) {
    clear_stale_error();
    if (!s || !a_c || !a_p) DECT_FAIL(DECT_EINVAL, "dect_forward_model: null argument");
    if (n < 0) DECT_FAIL(DECT_EINVAL, "dect_forward_model: n_rays < 0");
    if (dtype != DECT_F32 && dtype != DECT_F64) DECT_FAIL(DECT_EUNSUPPORTED, "dect_forward_model: bad dtype");
    launch_forward_model(s->dev(), s->t64, n, dtype, a_c, a_p, f_h, f_l, jac, nullptr, nullptr, nullptr, nullptr,
                         as_stream(stream));
    CUDA_TRY(cudaGetLastError());
    return DECT_OK;
}

extern "C" dect_status dect_forward_model_vjp(const dect_spectra* s, int64_t n, int32_t dtype, const void* a_c,
                                              const void* a_p, const void* g_h, const void* g_l, void* grad_c,
                                              void* grad_p, void* stream) {
    clear_stale_error();
    if (!s || !a_c || !a_p || !g_h || !g_l || !grad_c || !grad_p)
        DECT_FAIL(DECT_EINVAL, "dect_forward_model_vjp: null argument");
    if (n < 0) DECT_FAIL(DECT_EINVAL, "dect_forward_model_vjp: n_rays < 0");
    if (dtype != DECT_F32 && dtype != DECT_F64) DECT_FAIL(DECT_EUNSUPPORTED, "dect_forward_model_vjp: bad dtype");
    launch_forward_model(s->dev(), s->t64, n, dtype, a_c, a_p, nullptr, nullptr, nullptr, g_h, g_l, grad_c, grad_p,
                         as_stream(stream));
    CUDA_TRY(cudaGetLastError());
    return DECT_OK;
}

// ----------------------------------------------------------------------------------------------
extern "C" void dect_params_default(dect_params* p) {
    if (!p) return;
    p->lambda_c = 1e-5;
    p->lambda_p = 1e-5;
    p->rho0_c = 1e-3;
    p->rho0_p = 1e-3;
    p->m_udm = 1;
    p->n_pcg = 1;
    p->rho_mu = 10.0;
    p->rho_tau = 2.0;
    p->lm_mu0 = 1e-3;
    p->kappa = 1e-2;
    p->init_udm_iters = 10;
    p->init_pcg_iters = 10;
    p->precondition = DECT_PRECOND_CIRCULANT;
    p->use_graph = 1;
    p->bp_view_groups = 0;
    p->storage = DECT_STORE_F32;
    p->scheme = DECT_SCHEME_UDM_PCG;
    p->init = DECT_INIT_PCG;
    p->udm_f64 = 0;
    p->objective_every = 0;
    p->bp_tile = 0;
    p->bp_cluster = 0;
    p->bp_slices = 0;
    p->bp_reduce = 0;
    p->proj_views = 0;
}

struct MapBuf {
    int* d = nullptr;
    std::vector<int> h;  // B+1 prefix
    int total = 0;
    BlockMap map(int B) const { return BlockMap{d, B}; }
};

struct dect_admm {
    int B = 0;
    std::vector<dect_geom*> geoms;
    const dect_spectra* spec = nullptr;
    dect_params P{};
    std::vector<SliceDesc> hs;
    SliceDesc* ds = nullptr;
    MapBuf rays, pix, tx, ty, rows, cols, sweep, ptile;  // ptile: the projector's (views x bins) tiles per group
    MapBuf prows, pcols;  // the preconditioner apply's row and column blocks (split or staged, per slice)
    // row-block prefix of the <r, s> partials the float32 preconditioner wrote
    const int* rs_prefix() const { return P.precondition ? prows.d : rows.d; }
    int n_groups = 0;                // projector groups: consecutive slices of one geometry (proj_group_size())
    std::vector<int2> group_shape;   // {views, bins} per projector group
    int proj_views = 2;              // views per projector CTA (2, 4 or 8; does not change results)
    int4* d_groups = nullptr;        // {slice, further slices or -1} per group
    int sweep_C = 1;                 // CTA groups (partial images) per backprojector tile
    int sweep_tile = kSweepTileDefault;  // backprojector tile side (32 or 64; does not change results)
    bool sweep_cluster = false;      // the view groups of a tile reduce on chip into one partial image
    std::vector<int> cluster_cands;  // cluster forms the autotuner may time (0 off, 1 on)
    int sweep_sg = 1;                // slices per sweep CTA (2: pairs of consecutive slices of one geometry)
    std::vector<int> sg_cands;       // slices per CTA the autotuner may time
    std::vector<int4> sgroups;       // the pairs (second -1 for a slice without a partner)
    int4* d_sgroups = nullptr;
    int sweep_units() const { return sweep_sg == 2 ? (int)sgroups.size() : B; }
    bool sweep_reduce = false;       // the last CTA of a tile sums its C partials into image 0 (reduced form)
    int* tile_count = nullptr;       // the reduced form's arrival counters, one per tile (zero between launches)
    int n_tile_count = 0;            // counters: the batch's tiles at the smallest tile side
    int* reduce_count() const { return sweep_reduce && !sweep_cluster ? tile_count : nullptr; }
    int bp_slots() const { return sweep_cluster ? 1 : sweep_C; }  // partial images the sweep writes
    int bp_parts() const { return sweep_cluster || (sweep_reduce && sweep_C > 1) ? 1 : sweep_C; }  // the finalize reads
    int sweep_groups_in_use = 1;     // view groups per tile (sweep_C CTAs of the kernel's groups each)
    float2* bp_partial = nullptr;    // [sweep_C][n_img] partial images of the backprojector
    int64_t n_img = 0, n_sino = 0, n_tx = 0, n_ty = 0, n_fft = 0, n_h = 0, n_stage = 0;
    int max_px = 0, min_px = 1 << 30, min_py = 1 << 30;
    float2 *x = nullptr, *r = nullptr, *s = nullptr, *p = nullptr, *Ap = nullptr, *z = nullptr, *uz = nullptr;
    float2 *x0 = nullptr, *truth = nullptr, *Z = nullptr;
    void *Rx = nullptr, *a = nullptr, *ua = nullptr, *q = nullptr;  // sinogram vectors, storage format `prec`
    void *txb = nullptr, *tyb = nullptr;                            // pair textures, storage format `prec`
    float4 *y = nullptr, *uy = nullptr, *meas = nullptr;
    int prec = PREC_F32;
    float *mu = nullptr, *H = nullptr, *Hn = nullptr, *stage = nullptr;
    float *Hp = nullptr, *Hnp = nullptr;  // H and Hn permuted for the split column pass
    uint8_t* status = nullptr;
    SliceScalars* sc = nullptr;
    double *part_udm = nullptr, *part_img = nullptr, *part_rs = nullptr, *part_pap = nullptr, *part_xi = nullptr;
    // comparison scheme LM(m) x CG(n): per-slice scalars, single-channel CG vectors (d, r, p, A p), per-ray
    // Gauss-Newton weights (e, g), spectral sums at x (s0), R p (q1), carried R d, single-channel textures
    // and partial images, one partial slot per pixel / ray block
    LmScalars* ls = nullptr;
    float* lm_scale = nullptr;
    float *lm_d = nullptr, *lm_r = nullptr, *lm_p = nullptr, *lm_Ap = nullptr;
    float *lm_e = nullptr, *lm_g = nullptr, *lm_q = nullptr, *lm_Rd = nullptr;
    float2* lm_s0 = nullptr;
    float2 *tx1 = nullptr, *ty1 = nullptr;
    float* bp_partial1 = nullptr;
    double *part_lm_pix = nullptr, *part_lm_ray = nullptr;
    int* d_has_x0 = nullptr;
    // float64 path (storage DECT_STORE_F64): its vectors, a one-column-per-block FFT map and the slices'
    // float64 ray tables (owned by the geometries)
    F64Vecs v64;
    MapBuf cols64;
    int max_py = 0;
    std::vector<const double4_32a*> rays64;
    std::vector<int> has_x0, has_truth, has_data;
    const float2* tw = nullptr;
    bool initialized = false;
    bool counting = true;
    cudaStream_t cap = nullptr;
    cudaGraphExec_t gexec = nullptr;
    int64_t cR = 0, cRT = 0, cF = 0, cL = 0;
    int64_t iters_done = 0;                            // iterations since the last (re)initialisation
    double *part_obj_rays = nullptr, *part_obj_pix = nullptr;  // Eq. 4 partials (one per ray / pixel block)
    int64_t launches_per_iter = 0, R_per_iter = 0, RT_per_iter = 0, f_per_iter = 0;
    // profiling: an event pair around every kernel group of the captured iteration
    bool prof_on = false;
    int prof_n = 0;
    std::vector<cudaEvent_t> prof_ev;
    std::vector<int> prof_phase, prof_kernels;
    cudaGraphExec_t pgexec = nullptr;
};

static constexpr int kMaxProfGroups = 128;

// Marks the start of a kernel group (records an event when profiling is being captured).
static void pb(dect_admm* A, cudaStream_t st) {
    // external records: captured as event-record nodes of the graph (not only as dependencies)
    if (A->prof_on && A->prof_n < kMaxProfGroups)
        cudaEventRecordWithFlags(A->prof_ev[2 * A->prof_n], st, cudaEventRecordExternal);
}

// Marks the end of a group of `nk` kernels of `phase`; counts the launches.
static void pe(dect_admm* A, int phase, int nk, cudaStream_t st) {
    if (A->counting) A->cL += nk;
    if (A->prof_on && A->prof_n < kMaxProfGroups) {
        cudaEventRecordWithFlags(A->prof_ev[2 * A->prof_n + 1], st, cudaEventRecordExternal);
        A->prof_phase.push_back(phase);
        A->prof_kernels.push_back(nk);
        A->prof_n++;
    }
}

static void free_admm(dect_admm* A) {
    void* ptrs[] = {A->ds, A->rays.d, A->pix.d, A->tx.d, A->ty.d, A->rows.d, A->cols.d, A->sweep.d, A->ptile.d, A->d_groups,
                    A->d_sgroups,
                    A->bp_partial, A->x, A->r, A->s,
                    A->p, A->Ap, A->z, A->uz, A->x0, A->truth, A->Rx, A->a, A->ua, A->q, A->Z, A->y, A->uy,
                    A->meas, A->txb, A->tyb, A->mu, A->H, A->Hn, A->stage, A->status, A->sc, A->part_udm,
                    A->part_img, A->part_rs, A->part_pap, A->part_xi, A->d_has_x0, A->ls, A->lm_scale, A->lm_d,
                    A->lm_r, A->lm_p, A->lm_Ap, A->lm_e, A->lm_g, A->lm_q, A->lm_Rd, A->lm_s0, A->tx1, A->ty1,
                    A->bp_partial1, A->part_lm_pix, A->part_lm_ray, A->cols64.d, A->part_obj_rays,
                    A->part_obj_pix, A->tile_count, A->prows.d, A->pcols.d, A->Hp, A->Hnp};
    for (void* q : ptrs) cudaFree(q);
    const F64Vecs& v = A->v64;
    for (void* q : {(void*)v.x, (void*)v.r, (void*)v.s, (void*)v.p, (void*)v.Ap, (void*)v.z, (void*)v.uz, (void*)v.x0,
                    (void*)v.y, (void*)v.uy, (void*)v.RTs, (void*)v.Rx, (void*)v.a, (void*)v.ua, (void*)v.q,
                    (void*)v.mu, (void*)v.H, (void*)v.Hn, (void*)v.Z})
        cudaFree(q);
    if (A->gexec) cudaGraphExecDestroy(A->gexec);
    if (A->pgexec) cudaGraphExecDestroy(A->pgexec);
    for (cudaEvent_t e : A->prof_ev) cudaEventDestroy(e);
    if (A->cap) cudaStreamDestroy(A->cap);
    delete A;
}

// Device copy of a block map; capacity (entries) may exceed the current prefix when the map is later
// rewritten for another layout (the sweep's one-slice and slice-pair layouts).
static cudaError_t upload_map(MapBuf& m, size_t capacity = 0) {
    cudaError_t e = dalloc(&m.d, std::max(m.h.size(), capacity));
    if (e != cudaSuccess) return e;
    m.total = m.h.back();
    return cudaMemcpy(m.d, m.h.data(), sizeof(int) * m.h.size(), cudaMemcpyHostToDevice);
}

// ---- enqueue helpers ---------------------------------------------------------------------------

static void enq_project(dect_admm* A, const float2* img, void* out, cudaStream_t st) {
    const int B = A->B;
    pb(A, st);
    launch_textures(A->ds, A->tx.map(B), A->tx.total, A->ty.map(B), A->ty.total, img, A->txb, A->tyb, A->prec, st);
    pe(A, DECT_PHASE_TEXTURE, 2, st);
    pb(A, st);
    launch_project(A->ds, A->ptile.map(A->n_groups), A->ptile.total, A->d_groups, A->txb, A->tyb, out, A->prec,
                   A->proj_views, st);
    pe(A, DECT_PHASE_PROJECT, 1, st);
    if (A->counting) A->cR += 2;
}

static void enq_precond(dect_admm* A, const float* H, const float2* r, float2* s, cudaStream_t st) {
    const int B = A->B;
    pb(A, st);
    if (A->P.precondition) {
        launch_precond(A->ds, A->prows.map(B), A->prows.total, A->pcols.map(B), A->pcols.total, H,
                       H == A->H ? A->Hp : A->Hnp, r, s, A->Z, A->part_rs, A->tw, A->max_px, A->min_px, A->max_py,
                       A->min_py, st);
        pe(A, DECT_PHASE_PRECOND, 3, st);
    } else {
        launch_identity_precond(A->ds, A->rows.map(B), A->rows.total, r, s, A->part_rs, st);
        pe(A, DECT_PHASE_PRECOND, 1, st);
    }
}

// Eq. 12: n PCG steps, warm-started from x, R x carried
static void enq_pcg(dect_admm* A, int n, bool with_grad, const float* H, cudaStream_t st) {
    const int B = A->B;
    BpEpilogue ep{};
    ep.x = A->x;
    ep.y = A->y;
    ep.uy = A->uy;
    ep.z = A->z;
    ep.uz = A->uz;
    ep.p = A->p;
    ep.partial = A->part_pap;
    pb(A, st);
    launch_sino_resid(A->ds, A->rays.map(B), A->rays.total, A->a, A->ua, A->Rx, A->q, A->prec, st);
    pe(A, DECT_PHASE_UPDATE, 1, st);
    pb(A, st);
    launch_bp_sweep(A->ds, A->sweep.map(A->sweep_units()), A->sweep.total, A->sweep_C, A->sweep_tile, A->sweep_cluster,
                    A->sweep_sg, A->d_sgroups, A->q, A->bp_partial, A->n_img, A->prec, A->reduce_count(), st);
    pe(A, DECT_PHASE_BACKPROJECT, 1, st);
    pb(A, st);
    launch_bp_finalize(with_grad ? BP_R0 : BP_R0_NOGRAD, A->ds, A->pix.map(B), A->pix.total, A->bp_parts(),
                       A->bp_partial, A->n_img, A->r, ep, st);
    pe(A, DECT_PHASE_BP_FINALIZE, 1, st);
    if (A->counting) A->cRT += 2;
    enq_precond(A, H, A->r, A->p, st);
    pb(A, st);
    launch_rs_reduce(A->part_rs, A->rs_prefix(), A->sc, B, 1, st);
    pe(A, DECT_PHASE_REDUCE, 1, st);
    for (int it = 0; it < n; ++it) {
        enq_project(A, A->p, A->q, st);
        pb(A, st);
        launch_bp_sweep(A->ds, A->sweep.map(A->sweep_units()), A->sweep.total, A->sweep_C, A->sweep_tile, A->sweep_cluster,
                        A->sweep_sg, A->d_sgroups, A->q, A->bp_partial, A->n_img, A->prec, A->reduce_count(), st);
        pe(A, DECT_PHASE_BACKPROJECT, 1, st);
        pb(A, st);
        launch_bp_finalize(with_grad ? BP_AP : BP_AP_NOGRAD, A->ds, A->pix.map(B), A->pix.total, A->bp_parts(),
                           A->bp_partial, A->n_img, A->Ap, ep, st);
        pe(A, DECT_PHASE_BP_FINALIZE, 1, st);
        if (A->counting) A->cRT += 2;
        pb(A, st);
        launch_alpha(A->part_pap, A->pix.d, A->sc, B, st);
        pe(A, DECT_PHASE_REDUCE, 1, st);
        const int last = it == n - 1;
        pb(A, st);
        launch_cg_update(A->ds, A->pix.map(B), A->pix.total, A->rays.map(B), A->rays.total, A->sc, A->x, A->p, A->r,
                         A->Ap, A->Rx, A->q, last, A->prec, st);
        pe(A, DECT_PHASE_UPDATE, 1, st);
        if (!last) {
            enq_precond(A, H, A->r, A->s, st);
            pb(A, st);
            launch_rs_reduce(A->part_rs, A->rs_prefix(), A->sc, B, 0, st);
            pe(A, DECT_PHASE_REDUCE, 1, st);
            pb(A, st);
            launch_cg_p(A->ds, A->pix.map(B), A->pix.total, A->sc, A->s, A->p, st);
            pe(A, DECT_PHASE_UPDATE, 1, st);
        }
    }
}

// One LM step on basis b for every slice (Eq. 7 for b = 0, Eq. 8 for b = 1): Gauss-Newton weights, the
// gradient (one single-channel R^T), n CG iterations (one R and one R^T each; R d carried), the trial's
// objective change and the accept / damping decision, then x_b and (R x)_b move on accepted slices.
static void enq_lm_step(dect_admm* A, int b, cudaStream_t st) {
    const int B = A->B, n = A->P.n_pcg;
    const BlockMap pix = A->pix.map(B), rays = A->rays.map(B);
    BpEpilogue ep{};
    ep.x = A->x;
    ep.y = A->y;
    ep.uy = A->uy;
    ep.z = A->z;
    ep.uz = A->uz;
    pb(A, st);
    launch_lm_rays(A->ds, rays, A->rays.total, A->spec->dev(), A->meas, (const float2*)A->Rx, b, A->lm_e, A->lm_g,
                   A->lm_s0, A->lm_Rd, st);
    pe(A, DECT_PHASE_UDM, 1, st);
    pb(A, st);
    launch_bp_sweep1(A->ds, A->sweep.map(B), A->sweep.total, A->sweep_C, A->sweep_tile, A->sweep_cluster, A->lm_e,
                     nullptr, nullptr, A->bp_partial1, A->n_img, A->reduce_count(), st);
    pe(A, DECT_PHASE_BACKPROJECT, 1, st);
    pb(A, st);
    launch_lm_grad(A->ds, pix, A->pix.total, A->bp_parts(), A->bp_partial1, A->n_img, b, A->sc, ep, A->lm_r, A->lm_p,
                   A->lm_d, A->part_lm_pix, st);
    pe(A, DECT_PHASE_BP_FINALIZE, 1, st);
    pb(A, st);
    launch_lm_rr(A->part_lm_pix, A->pix.d, A->ls, B, 1, st);
    pe(A, DECT_PHASE_REDUCE, 1, st);
    if (A->counting) A->cRT += 1;
    for (int k = 0; k < n; ++k) {
        const int last = k == n - 1;
        pb(A, st);
        launch_textures1(A->ds, A->tx.map(B), A->tx.total, A->ty.map(B), A->ty.total, A->lm_p, A->tx1, A->ty1, st);
        pe(A, DECT_PHASE_TEXTURE, 2, st);
        pb(A, st);
        launch_project1(A->ds, A->ptile.map(A->n_groups), A->ptile.total, A->d_groups, A->tx1, A->ty1, A->lm_q,
                        A->proj_views, st);
        pe(A, DECT_PHASE_PROJECT, 1, st);
        pb(A, st);
        launch_bp_sweep1(A->ds, A->sweep.map(B), A->sweep.total, A->sweep_C, A->sweep_tile, A->sweep_cluster, A->lm_q,
                         A->lm_g, A->lm_scale, A->bp_partial1, A->n_img, A->reduce_count(), st);
        pe(A, DECT_PHASE_BACKPROJECT, 1, st);
        pb(A, st);
        launch_lm_ap(A->ds, pix, A->pix.total, A->bp_parts(), A->bp_partial1, A->n_img, b, A->sc, A->lm_p, A->lm_Ap,
                     A->part_lm_pix, st);
        pe(A, DECT_PHASE_BP_FINALIZE, 1, st);
        pb(A, st);
        launch_lm_alpha(A->part_lm_pix, A->pix.d, A->ls, B, st);
        pe(A, DECT_PHASE_REDUCE, 1, st);
        pb(A, st);
        launch_lm_cg(A->ds, pix, A->pix.total, rays, A->rays.total, A->ls, A->lm_d, A->lm_p, A->lm_r, A->lm_Ap,
                     A->lm_Rd, A->lm_q, last, A->part_lm_pix, st);
        pe(A, DECT_PHASE_UPDATE, 1, st);
        if (A->counting) {
            A->cR += 1;
            A->cRT += 1;
        }
        if (!last) {
            pb(A, st);
            launch_lm_rr(A->part_lm_pix, A->pix.d, A->ls, B, 0, st);
            pe(A, DECT_PHASE_REDUCE, 1, st);
            pb(A, st);
            launch_lm_p(A->ds, pix, A->pix.total, A->ls, A->lm_r, A->lm_p, st);
            pe(A, DECT_PHASE_UPDATE, 1, st);
        }
    }
    pb(A, st);
    launch_lm_trial(A->ds, rays, A->rays.total, A->spec->dev(), A->meas, (const float2*)A->Rx, b, A->lm_Rd, A->lm_s0,
                    A->part_lm_ray, st);
    pe(A, DECT_PHASE_UDM, 1, st);
    pb(A, st);
    launch_lm_al_delta(A->ds, pix, A->pix.total, b, A->sc, ep, A->lm_d, A->part_lm_pix, st);
    pe(A, DECT_PHASE_UPDATE, 1, st);
    pb(A, st);
    launch_lm_decide(A->part_lm_ray, A->rays.d, A->part_lm_pix, A->pix.d, A->ls, A->lm_scale, B, b, st);
    pe(A, DECT_PHASE_REDUCE, 1, st);
    pb(A, st);
    launch_lm_accept(A->ds, pix, A->pix.total, rays, A->rays.total, A->ls, b, A->x, A->lm_d, (float2*)A->Rx, A->lm_Rd,
                     st);
    pe(A, DECT_PHASE_UPDATE, 1, st);
    if (A->counting) A->cF += 2;
}

// One ADMM iteration of the comparison scheme: m LM steps on x_c, then on x_p (Eq. 7-8), then Eq. 9-11
// (no a-block: its residual slots stay zero) and residual-balancing rho.
static void enq_lmcg_iteration(dect_admm* A, cudaStream_t st) {
    const int B = A->B;
    for (int b = 0; b < 2; ++b) {
        pb(A, st);
        launch_lm_begin(A->ls, A->lm_scale, B, b, st);
        pe(A, DECT_PHASE_REDUCE, 1, st);
        for (int it = 0; it < A->P.m_udm; ++it) enq_lm_step(A, b, st);
    }
    pb(A, st);
    launch_image_update(A->ds, A->pix.map(B), A->pix.total, A->sc, A->P.lambda_c, A->P.lambda_p, A->x, A->y, A->uy,
                        A->z, A->uz, A->part_img, st);
    pe(A, DECT_PHASE_UPDATE, 1, st);
    pb(A, st);
    launch_rho_update(A->part_udm, A->rays.d, A->part_img, A->pix.d, A->sc, B, A->P.rho_mu, A->P.rho_tau, st);
    pe(A, DECT_PHASE_REDUCE, 1, st);
    pb(A, st);
    launch_dual_rescale(A->ds, B, A->sc, A->uy, A->uz, A->ua,
                        A->prec, st);
    pe(A, DECT_PHASE_UPDATE, 1, st);
}

// ---- float64 path (storage DECT_STORE_F64): the same iteration with float64 kernels ----------------

static void enq_project64(dect_admm* A, const double* img, double* out, cudaStream_t st) {
    pb(A, st);
    for (int b = 0; b < A->B; ++b) {
        const SliceDesc& sd = A->hs[b];
        project_single_f64(sd.g, A->rays64[b], img + 2 * sd.img_off, 2, out + 2 * sd.sino_off, st);
    }
    pe(A, DECT_PHASE_PROJECT, A->B, st);
    if (A->counting) A->cR += 2;
}

static void enq_backproject64(dect_admm* A, const double* sino, double* out, cudaStream_t st) {
    pb(A, st);
    for (int b = 0; b < A->B; ++b) {
        const SliceDesc& sd = A->hs[b];
        backproject_single_f64(sd.g, A->rays64[b], sino + 2 * sd.sino_off, 2, out + 2 * sd.img_off, st);
    }
    pe(A, DECT_PHASE_BACKPROJECT, A->B, st);
    if (A->counting) A->cRT += 2;
}

static void enq_precond64(dect_admm* A, const double* H, const double* r, double* s, cudaStream_t st) {
    const int B = A->B;
    const double* h = A->P.precondition ? H : nullptr;
    pb(A, st);
    launch64_precond(A->ds, A->rows.map(B), A->rows.total, A->cols64.map(B), A->cols64.total, h, r, s, A->v64.Z,
                     A->part_rs, A->max_px, A->max_py, st);
    pe(A, DECT_PHASE_PRECOND, h ? 3 : 1, st);
}

// Eq. 12 in float64: n PCG steps, warm-started from x, R x carried
static void enq_pcg64(dect_admm* A, int n, bool with_grad, const double* H, cudaStream_t st) {
    const int B = A->B;
    F64Vecs& v = A->v64;
    const BlockMap pix = A->pix.map(B), rays = A->rays.map(B);
    pb(A, st);
    launch64_sino_resid(A->ds, rays, A->rays.total, v.a, v.ua, v.Rx, v.q, st);
    pe(A, DECT_PHASE_UPDATE, 1, st);
    enq_backproject64(A, v.q, v.RTs, st);
    pb(A, st);
    launch64_r0(A->ds, pix, A->pix.total, v.RTs, v, v.r, with_grad, st);
    pe(A, DECT_PHASE_BP_FINALIZE, 1, st);
    enq_precond64(A, H, v.r, v.p, st);
    pb(A, st);
    launch_rs_reduce(A->part_rs, A->rows.d, A->sc, B, 1, st);
    pe(A, DECT_PHASE_REDUCE, 1, st);
    for (int it = 0; it < n; ++it) {
        enq_project64(A, v.p, v.q, st);
        enq_backproject64(A, v.q, v.RTs, st);
        pb(A, st);
        launch64_ap(A->ds, pix, A->pix.total, v.RTs, v.p, v.Ap, A->part_pap, with_grad, st);
        pe(A, DECT_PHASE_BP_FINALIZE, 1, st);
        pb(A, st);
        launch_alpha(A->part_pap, A->pix.d, A->sc, B, st);
        pe(A, DECT_PHASE_REDUCE, 1, st);
        const int last = it == n - 1;
        pb(A, st);
        launch64_cg_update(A->ds, pix, A->pix.total, rays, A->rays.total, A->sc, v, last, st);
        pe(A, DECT_PHASE_UPDATE, 1, st);
        if (!last) {
            enq_precond64(A, H, v.r, v.s, st);
            pb(A, st);
            launch_rs_reduce(A->part_rs, A->rows.d, A->sc, B, 0, st);
            pe(A, DECT_PHASE_REDUCE, 1, st);
            pb(A, st);
            launch64_cg_p(A->ds, pix, A->pix.total, A->sc, v.s, v.p, st);
            pe(A, DECT_PHASE_UPDATE, 1, st);
        }
    }
}

static void enq_iteration64(dect_admm* A, cudaStream_t st) {
    const int B = A->B;
    F64Vecs& v = A->v64;
    const BlockMap pix = A->pix.map(B), rays = A->rays.map(B);
    enq_pcg64(A, A->P.n_pcg, true, v.H, st);
    pb(A, st);
    launch64_udm_admm(A->ds, rays, A->rays.total, A->spec->t64, A->spec->ne, A->meas, v, A->status, A->sc,
                      A->P.m_udm, A->part_udm, st);
    pe(A, DECT_PHASE_UDM, 1, st);
    if (A->counting) A->cF += 4 * A->P.m_udm;
    pb(A, st);
    launch64_image_update(A->ds, pix, A->pix.total, A->sc, A->P.lambda_c, A->P.lambda_p, v, A->part_img, st);
    pe(A, DECT_PHASE_UPDATE, 1, st);
    pb(A, st);
    launch_rho_update(A->part_udm, A->rays.d, A->part_img, A->pix.d, A->sc, B, A->P.rho_mu, A->P.rho_tau, st);
    pe(A, DECT_PHASE_REDUCE, 1, st);
    pb(A, st);
    launch64_dual_rescale(A->ds, pix, A->pix.total, rays, A->rays.total, A->sc, v, st);
    pe(A, DECT_PHASE_UPDATE, 1, st);
}

static void enq_iteration(dect_admm* A, cudaStream_t st) {
    const int B = A->B;
    if (A->prec == PREC_F64) {
        enq_iteration64(A, st);
        return;
    }
    if (A->P.scheme == DECT_SCHEME_LM_CG) {
        enq_lmcg_iteration(A, st);
        return;
    }
    enq_pcg(A, A->P.n_pcg, true, A->H, st);
    pb(A, st);
    launch_udm_admm(A->ds, A->rays.map(B), A->rays.total, A->spec->dev(), A->meas, A->Rx, A->ua, A->a, A->mu,
                    A->status, A->sc, A->P.m_udm, A->part_udm, A->prec, A->P.udm_f64 != 0, st);
    pe(A, DECT_PHASE_UDM, 1, st);
    if (A->counting) A->cF += 4 * A->P.m_udm;
    pb(A, st);
    launch_image_update(A->ds, A->pix.map(B), A->pix.total, A->sc, A->P.lambda_c, A->P.lambda_p, A->x, A->y, A->uy,
                        A->z, A->uz, A->part_img, st);
    pe(A, DECT_PHASE_UPDATE, 1, st);
    pb(A, st);
    launch_rho_update(A->part_udm, A->rays.d, A->part_img, A->pix.d, A->sc, B, A->P.rho_mu, A->P.rho_tau, st);
    pe(A, DECT_PHASE_REDUCE, 1, st);
    pb(A, st);
    launch_dual_rescale(A->ds, B, A->sc, A->uy, A->uz, A->ua,
                        A->prec, st);
    pe(A, DECT_PHASE_UPDATE, 1, st);
}

// Eq. 4 at the current x of every slice: a fresh projection R x, the data term per ray and the TV
// term per pixel, summed per slice into the scalars (objective, and the iteration it belongs to).
// A monitor: its projection is not one of Table 1's applications (cR is left as it was).
static void enq_objective(dect_admm* A, cudaStream_t st) {
    const int B = A->B;
    const BlockMap pix = A->pix.map(B), rays = A->rays.map(B);
    const int64_t r0 = A->cR;
    if (A->prec == PREC_F64) {
        enq_project64(A, A->v64.x, A->v64.q, st);
        launch64_objective(A->ds, rays, A->rays.total, pix, A->pix.total, A->spec->t64, A->spec->ne, A->meas,
                           A->v64.q, A->v64.x, A->P.lambda_c, A->P.lambda_p, A->part_obj_rays, A->part_obj_pix, st);
    } else {
        enq_project(A, A->x, A->q, st);
        launch_objective_rays(A->ds, rays, A->rays.total, A->spec->dev(), A->meas, A->q, A->part_obj_rays, A->prec,
                              st);
        launch_objective_tv(A->ds, pix, A->pix.total, A->x, A->P.lambda_c, A->P.lambda_p, A->part_obj_pix, st);
    }
    launch_objective_reduce(A->part_obj_rays, A->rays.d, A->part_obj_pix, A->pix.d, A->sc, B, st);
    A->cR = r0;
    A->cL += 3;
}

// Captures one iteration into a graph (with event pairs when profiling).
static dect_status capture_iteration(dect_admm* A, bool profile, cudaGraphExec_t* out) {
    cudaGraph_t graph = nullptr;
    A->counting = false;
    A->prof_on = profile;
    A->prof_n = 0;
    A->prof_phase.clear();
    A->prof_kernels.clear();
    const int64_t l0 = A->cL;
    cudaError_t e = cudaStreamBeginCapture(A->cap, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        A->counting = true;  // count launches of one iteration, then restore the other counters
        const int64_t r0 = A->cR, rt0 = A->cRT, f0 = A->cF;
        enq_iteration(A, A->cap);
        A->launches_per_iter = A->cL - l0;
        A->R_per_iter = A->cR - r0;
        A->RT_per_iter = A->cRT - rt0;
        A->f_per_iter = A->cF - f0;
        A->cL = l0;
        A->cR = r0;
        A->cRT = rt0;
        A->cF = f0;
        e = cudaStreamEndCapture(A->cap, &graph);
    }
    A->counting = true;
    A->prof_on = false;
    CUDA_TRY(e);
    e = cudaGraphInstantiate(out, graph, 0);
    cudaGraphDestroy(graph);
    CUDA_TRY(e);
    return DECT_OK;
}

// The paper's start (Sec. 4): x_c of the slices without x0 = the Compton image of CDM-FBP (per-ray
// decomposition with rho = 0, a >= 0, FBP); k_init_image then clamps it and sets x_p = kappa x_c.
static dect_status enq_cdm_fbp_start(dect_admm* A, cudaStream_t st) {
    int64_t max_nr = 0;
    for (int b = 0; b < A->B; ++b) max_nr = std::max(max_nr, (int64_t)A->hs[b].g.nv * A->hs[b].g.nb);
    float* work = nullptr;  // a_c, a_p, mu, zeros of one slice
    CUDA_TRY(cudaMallocAsync((void**)&work, sizeof(float) * 4 * (size_t)max_nr, st));
    dect_status status = DECT_OK;
    for (int b = 0; b < A->B && status == DECT_OK; ++b) {
        if (A->has_x0[b]) continue;
        const SliceDesc& sd = A->hs[b];
        const int64_t nr = (int64_t)sd.g.nv * sd.g.nb, np = (int64_t)sd.g.nx * sd.g.ny;
        FbpDev f{};
        status = fbp_prepare(A->geoms[b], f);
        if (status != DECT_OK) break;
        float* m = A->stage;          // planar m_h, m_l, w_h, w_l
        float* img = A->stage + 4 * nr;  // planar [2][ny][nx]: Compton, then zeros
        launch_unpack_meas(nr, A->meas + sd.sino_off, m, st);
        launch_cdm_start(nr, m + nr, (float)(1.0 / A->spec->abar_low), (float)A->P.lm_mu0, work, work + nr,
                         work + 2 * nr, work + 3 * nr, st);
        launch_udm_rays(A->spec->dev(), nr, m, m + nr, m + 2 * nr, m + 3 * nr, work + 3 * nr, work + 3 * nr, 0.0,
                        0.0, A->P.init_udm_iters, work, work + nr, work + 2 * nr, nullptr, st);
        launch_fbp(f, 1, work, A->geoms[b]->fbp_q, img, true, st);
        cudaError_t e = cudaMemsetAsync(img + np, 0, sizeof(float) * np, st);
        if (e != cudaSuccess) {
            status = DECT_ECUDA;
            dect::set_error(std::string("dect_admm init: ") + cudaGetErrorString(e));
            break;
        }
        launch_interleave(img, np, A->x + sd.img_off, st);
    }
    A->cF += 4 * A->P.init_udm_iters;
    cudaError_t fe = cudaFreeAsync(work, st);
    if (status != DECT_OK) return status;
    CUDA_TRY(fe);
    return DECT_OK;
}

// The float64 path's start (the same steps as enq_initialize below, DECT_INIT_PCG only).
static dect_status enq_initialize64(dect_admm* A, bool all_x0, cudaStream_t st) {
    const int B = A->B;
    F64Vecs& v = A->v64;
    const BlockMap pix = A->pix.map(B), rays = A->rays.map(B);
    const size_t ni = (size_t)A->n_img, ns = (size_t)A->n_sino;
    if (!all_x0) {
        CUDA_TRY(cudaMemsetAsync(v.x, 0, sizeof(double) * 2 * ni, st));
        CUDA_TRY(cudaMemsetAsync(v.Rx, 0, sizeof(double) * 2 * ns, st));
        CUDA_TRY(cudaMemsetAsync(v.ua, 0, sizeof(double) * 2 * ns, st));
        CUDA_TRY(cudaMemsetAsync(v.y, 0, sizeof(double) * 4 * ni, st));
        CUDA_TRY(cudaMemsetAsync(v.uy, 0, sizeof(double) * 4 * ni, st));
        CUDA_TRY(cudaMemsetAsync(v.z, 0, sizeof(double) * 2 * ni, st));
        CUDA_TRY(cudaMemsetAsync(v.uz, 0, sizeof(double) * 2 * ni, st));
        launch64_udm_init(A->ds, rays, A->rays.total, A->spec->t64, A->spec->ne, A->meas, v, A->P.rho0_p,
                          A->P.init_udm_iters, A->spec->abar_low, A->P.lm_mu0, st);
        A->cF += 4 * A->P.init_udm_iters;
        launch_reset_scalars(A->sc, B, A->P.rho0_c, A->P.rho0_p, st);
        enq_pcg64(A, A->P.init_pcg_iters, false, v.Hn, st);
    }
    launch64_init_image(A->ds, pix, A->pix.total, A->d_has_x0, v, A->P.kappa, st);
    enq_project64(A, v.x, v.Rx, st);
    launch64_state_from_image(A->ds, pix, A->pix.total, rays, A->rays.total, v, A->P.lm_mu0, st);
    launch_reset_scalars(A->sc, B, A->P.rho0_c, A->P.rho0_p, st);
    CUDA_TRY(cudaGetLastError());
    A->iters_done = 0;
    A->initialized = true;
    return DECT_OK;
}

static dect_status enq_initialize(dect_admm* A, cudaStream_t st) {
    const int B = A->B;
    for (int b = 0; b < B; ++b)
        if (!A->has_data[b]) DECT_FAIL(DECT_EINVAL, "dect_admm: slice " + std::to_string(b) + " has no data");
    CUDA_TRY(cudaMemcpyAsync(A->d_has_x0, A->has_x0.data(), sizeof(int) * B, cudaMemcpyHostToDevice, st));
    if (A->prec == PREC_F64) {
        bool all = true;
        for (int b = 0; b < B; ++b) all = all && A->has_x0[b];
        return enq_initialize64(A, all, st);
    }
    bool all_x0 = true;
    for (int b = 0; b < B; ++b) all_x0 = all_x0 && A->has_x0[b];
    if (!all_x0) {
        CUDA_TRY(cudaMemsetAsync(A->x, 0, sizeof(float2) * A->n_img, st));
        CUDA_TRY(cudaMemsetAsync(A->Rx, 0, sino_bytes(A->prec) * A->n_sino, st));
        CUDA_TRY(cudaMemsetAsync(A->ua, 0, sino_bytes(A->prec) * A->n_sino, st));
        CUDA_TRY(cudaMemsetAsync(A->y, 0, sizeof(float4) * A->n_img, st));
        CUDA_TRY(cudaMemsetAsync(A->uy, 0, sizeof(float4) * A->n_img, st));
        CUDA_TRY(cudaMemsetAsync(A->z, 0, sizeof(float2) * A->n_img, st));
        CUDA_TRY(cudaMemsetAsync(A->uz, 0, sizeof(float2) * A->n_img, st));
        if (A->P.init == DECT_INIT_CDM_FBP) {
            const dect_status s = enq_cdm_fbp_start(A, st);
            if (s != DECT_OK) return s;
        } else {
            launch_udm_init(A->ds, A->rays.map(B), A->rays.total, A->spec->dev(), A->meas, A->a, A->mu,
                            A->P.rho0_p, A->P.init_udm_iters, (float)A->spec->abar_low, A->P.lm_mu0, A->prec, st);
            A->cF += 4 * A->P.init_udm_iters;
            launch_reset_scalars(A->sc, B, A->P.rho0_c, A->P.rho0_p, st);
            enq_pcg(A, A->P.init_pcg_iters, false, A->Hn, st);
        }
    }
    launch_init_image(A->ds, A->pix.map(B), A->pix.total, A->d_has_x0, A->x0, A->x, (float)A->P.kappa, st);
    enq_project(A, A->x, A->Rx, st);
    launch_state_from_image(A->ds, A->pix.map(B), A->pix.total, A->rays.map(B), A->rays.total, A->x, A->y, A->uy,
                            A->z, A->uz, A->Rx, A->a, A->ua, A->mu, (float)A->P.lm_mu0, A->prec, st);
    launch_reset_scalars(A->sc, B, A->P.rho0_c, A->P.rho0_p, st);
    if (A->P.scheme == DECT_SCHEME_LM_CG) launch_lm_reset(A->ls, B, A->P.lm_mu0, st);
    CUDA_TRY(cudaGetLastError());
    A->iters_done = 0;
    A->initialized = true;
    return DECT_OK;
}

// ---- creation ------------------------------------------------------------------------------------

// Sweep block map for C CTA groups per TILE x TILE tile (prefix over slices, or over slice pairs for sg = 2)
static void sweep_prefix(const dect_admm* A, int C, int tile, int sg, std::vector<int>& h) {
    h.assign(1, 0);
    if (sg == 2)
        for (const int4& p : A->sgroups)
            h.push_back(h.back() + sweep_tiles(A->hs[p.x].g.nx, A->hs[p.x].g.ny, tile) * C);
    else
        for (int b = 0; b < A->B; ++b) h.push_back(h.back() + sweep_tiles(A->hs[b].g.nx, A->hs[b].g.ny, tile) * C);
}

// the projector's tile prefix over the geometry groups for `views` views per CTA
static void ptile_prefix(const dect_admm* A, int views, std::vector<int>& h) {
    h.assign(1, 0);
    for (const int2& g : A->group_shape) h.push_back(h.back() + proj_tiles(g.x, g.y, views));
}

// Times the forward projector on this batch for 2, 4 and 8 views per CTA (on the current textures; the
// work does not depend on the values) and keeps the fastest (fewer views unless more are 1% faster).
// Every choice gives the same bits. The tile map is rewritten for the choice.
static cudaError_t autotune_projector(dect_admm* A) {
    cudaStream_t st = A->cap;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    int best = A->proj_views;
    float best_ms = 0.f;
    bool first = true;
    std::vector<int> h;
    for (int views : {2, 4, 8}) {
        if (e != cudaSuccess) break;
        ptile_prefix(A, views, h);
        e = cudaMemcpy(A->ptile.d, h.data(), sizeof(int) * h.size(), cudaMemcpyHostToDevice);
        const BlockMap m{A->ptile.d, A->n_groups};
        auto run = [&]() { launch_project(A->ds, m, h.back(), A->d_groups, A->txb, A->tyb, A->q, A->prec, views, st); };
        run();  // warm-up
        e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaEventRecord(e0, st);
        for (int r = 0; r < 3 && e == cudaSuccess; ++r) {
            run();
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = cudaEventRecord(e1, st);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e == cudaSuccess && (first || ms < 0.99f * best_ms)) {
            best = views;
            best_ms = ms;
            first = false;
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (e != cudaSuccess) return e;
    A->proj_views = best;
    ptile_prefix(A, best, A->ptile.h);
    A->ptile.total = A->ptile.h.back();
    return cudaMemcpy(A->ptile.d, A->ptile.h.data(), sizeof(int) * A->ptile.h.size(), cudaMemcpyHostToDevice);
}

// Times the backprojector sweep on this batch (on a zero sinogram; the work does not depend on the
// values) and keeps the fastest shape (fewer view groups unless more are 1% faster), in three stages:
// slices per CTA x view groups C at the default tile side, then the other tile sides at the best of
// those, then the cluster form there. Shrinks the partial-image buffer to the choice (bp_partial is
// allocated for the largest candidate C). The tile side, the slices per CTA and the cluster form do
// not change results; C fixes the order of a pixel's partial sums.
static cudaError_t autotune_sweep(dect_admm* A, const std::vector<int>& cands, const std::vector<int>& tiles) {
    cudaStream_t st = A->cap;
    cudaError_t e = cudaMemsetAsync(A->q, 0, sino_bytes(A->prec) * (size_t)A->n_sino, st);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    const int tile0 =
        std::find(tiles.begin(), tiles.end(), kSweepTileDefault) != tiles.end() ? kSweepTileDefault : tiles[0];
    const bool cl0 = A->cluster_cands.size() == 1 && A->cluster_cands[0] == 1;  // cluster form required
    int best = cands[0], best_tile = tile0, best_sg = 1;
    bool best_cluster = false;
    float best_ms = 0.f;
    bool first = true;
    std::vector<int> h;
    auto trial = [&](int sg, int tile, int C, bool cluster) {
        if (e != cudaSuccess || (cluster && (C < 2 || C > 16 || sg != 1))) return;
        sweep_prefix(A, C, tile, sg, h);
        e = cudaMemcpy(A->sweep.d, h.data(), sizeof(int) * h.size(), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return;
        const BlockMap m{A->sweep.d, sg == 2 ? (int)A->sgroups.size() : A->B};
        auto run = [&]() {
            launch_bp_sweep(A->ds, m, h.back(), C, tile, cluster, sg, A->d_sgroups, A->q, A->bp_partial, A->n_img,
                            A->prec, A->sweep_reduce ? A->tile_count : nullptr, st);
        };
        // a cluster shape the device cannot schedule is reported at launch: skip that candidate
        run();
        if (cluster && cudaGetLastError() != cudaSuccess) return;
        run();  // warm-up
        e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaEventRecord(e0, st);
        for (int r = 0; r < 3 && e == cudaSuccess; ++r) {
            run();
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = cudaEventRecord(e1, st);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e == cudaSuccess && (first || ms < 0.99f * best_ms || (ms <= best_ms && C < best))) {
            best = C;
            best_tile = tile;
            best_cluster = cluster;
            best_sg = sg;
            best_ms = ms;
            first = false;
        }
    };
    for (int sg : A->sg_cands)
        for (int C : cands) trial(sg, tile0, C, cl0);
    const int C1 = best, sg1 = best_sg;
    const bool cl1 = best_cluster;
    for (int tile : tiles)
        if (tile != tile0) trial(sg1, tile, C1, cl1);
    if (A->cluster_cands.size() > 1) trial(1, best_tile, C1, true);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (e != cudaSuccess) return e;
    A->sweep_C = best;
    A->sweep_tile = best_tile;
    A->sweep_cluster = best_cluster;
    A->sweep_sg = best_sg;
    sweep_prefix(A, best, best_tile, best_sg, A->sweep.h);
    A->sweep.total = A->sweep.h.back();
    e = cudaMemcpy(A->sweep.d, A->sweep.h.data(), sizeof(int) * A->sweep.h.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return e;
    cudaFree(A->bp_partial);
    A->bp_partial = nullptr;
    e = dalloc(&A->bp_partial, (size_t)A->bp_slots() * A->n_img);
    return e;
}

// The float64 preconditioner responses: the point response of R^T R through the float64 projector
// pair, its 2D DFT in float64 and H (and H without D) from it.
static dect_status compute_responses64(dect_admm* A) {
    cudaStream_t st = A->cap;
    F64Vecs& v = A->v64;
    for (int b = 0; b < A->B; ++b) {
        const SliceDesc& sd = A->hs[b];
        const int64_t np = (int64_t)sd.g.nx * sd.g.ny;
        double* imp = v.r + 2 * sd.img_off;
        CUDA_TRY(cudaMemsetAsync(imp, 0, sizeof(double) * np, st));
        const double one = 1.0;
        const int64_t c = (int64_t)(sd.g.ny / 2) * sd.g.nx + sd.g.nx / 2;
        CUDA_TRY(cudaMemcpyAsync(imp + c, &one, sizeof(double), cudaMemcpyHostToDevice, st));
        project_single_f64(sd.g, A->rays64[b], imp, 1, v.q + 2 * sd.sino_off, st);
        backproject_single_f64(sd.g, A->rays64[b], v.q + 2 * sd.sino_off, 1, v.s + 2 * sd.img_off, st);
        SliceDesc one_slice = sd;
        one_slice.fft_off = 0;
        one_slice.h_off = 0;
        SliceDesc* dd = nullptr;
        int* pre = nullptr;
        CUDA_TRY(dalloc(&dd, 1));
        cudaError_t e = dalloc(&pre, 2);
        const int hp[2] = {0, sd.px};
        if (e == cudaSuccess) e = cudaMemcpyAsync(dd, &one_slice, sizeof(SliceDesc), cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(pre, hp, sizeof(hp), cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess) {
            launch64_response(dd, one_slice, BlockMap{pre, 1}, sd.px, v.s + 2 * sd.img_off, v.Z + sd.fft_off,
                              v.H + sd.h_off, v.Hn + sd.h_off, A->P.precondition == DECT_PRECOND_RAMP, st);
            e = cudaStreamSynchronize(st);
        }
        cudaFree(dd);
        cudaFree(pre);
        CUDA_TRY(e);
    }
    CUDA_TRY(cudaGetLastError());
    return DECT_OK;
}

static dect_status compute_responses(dect_admm* A) {
    if (A->prec == PREC_F64) return compute_responses64(A);
    cudaStream_t st = A->cap;
    for (int b = 0; b < A->B; ++b) {
        const SliceDesc& sd = A->hs[b];
        const int64_t np = (int64_t)sd.g.nx * sd.g.ny, nr = (int64_t)sd.g.nv * sd.g.nb;
        // unit impulse at pixel (ny/2, nx/2) in both channels
        CUDA_TRY(cudaMemsetAsync(A->stage, 0, sizeof(float) * 2 * np, st));
        const float one[1] = {1.0f};
        const int64_t c = (int64_t)(sd.g.ny / 2) * sd.g.nx + sd.g.nx / 2;
        CUDA_TRY(cudaMemcpyAsync(A->stage + c, one, sizeof(float), cudaMemcpyHostToDevice, st));
        CUDA_TRY(cudaMemcpyAsync(A->stage + np + c, one, sizeof(float), cudaMemcpyHostToDevice, st));
        CUDA_TRY(cudaStreamSynchronize(st));
        // float32 projector pair through the geometry's own workspace (independent of the storage format)
        dect_geom* g = A->geoms[b];
        dect_status ws = geom_workspace(g);
        if (ws != DECT_OK) return ws;
        project_single(sd, A->stage, 2, g->ws_img, g->ws_tx, g->ws_ty, A->stage + 2 * np, st);
        backproject_single(sd, g->ws_desc, g->ws_maps, g->ws_C, kSweepTileDefault, A->stage + 2 * np, 2, g->ws_sino,
                           g->ws_partial, A->stage, st);
        launch_interleave(A->stage, np, A->r + sd.img_off, st);
        // one-slice descriptor and column map
        SliceDesc one_slice = sd;
        one_slice.fft_off = 0;
        one_slice.h_off = 0;
        const int C = precond_cols_per_block(sd.py);
        const int ncols = (sd.px + C - 1) / C;
        SliceDesc* dd = nullptr;
        int* pre = nullptr;
        CUDA_TRY(dalloc(&dd, 1));
        CUDA_TRY(dalloc(&pre, 2));
        const int hp[2] = {0, ncols};
        CUDA_TRY(cudaMemcpyAsync(dd, &one_slice, sizeof(SliceDesc), cudaMemcpyHostToDevice, st));
        CUDA_TRY(cudaMemcpyAsync(pre, hp, sizeof(hp), cudaMemcpyHostToDevice, st));
        launch_psf_to_response(dd, one_slice, BlockMap{pre, 1}, ncols, A->r + sd.img_off, A->Z + sd.fft_off,
                               A->H + sd.h_off, A->Hn + sd.h_off, A->tw, A->P.precondition == DECT_PRECOND_RAMP,
                               st);
        launch_permute_response(sd, A->H, A->Hp, st);
        launch_permute_response(sd, A->Hn, A->Hnp, st);
        cudaError_t e = cudaStreamSynchronize(st);
        cudaFree(dd);
        cudaFree(pre);
        CUDA_TRY(e);
        (void)nr;
    }
    CUDA_TRY(cudaGetLastError());
    return DECT_OK;
}

extern "C" dect_status dect_admm_create(dect_geom* const* geoms, int32_t B, const dect_spectra* spec,
                                        const dect_params* P, dect_admm** out) {
    clear_stale_error();
    if (!geoms || !spec || !P || !out) DECT_FAIL(DECT_EINVAL, "dect_admm_create: null argument");
    *out = nullptr;
    if (B < 1 || B > 4096) DECT_FAIL(DECT_EINVAL, "dect_admm_create: n_slices must be in [1, 4096]");
    if (P->storage != DECT_STORE_F32 && P->storage != DECT_STORE_F16 && P->storage != DECT_STORE_BF16 &&
        P->storage != DECT_STORE_F64)
        DECT_FAIL(DECT_EINVAL, "dect_admm_create: storage must be DECT_STORE_F32, F16, BF16 or F64");
    if (P->udm_f64 != 0 && P->udm_f64 != 1) DECT_FAIL(DECT_EINVAL, "dect_admm_create: udm_f64 must be 0 or 1");
    if (P->objective_every < 0) DECT_FAIL(DECT_EINVAL, "dect_admm_create: objective_every must be >= 0");
    if (P->storage == DECT_STORE_F64) {
        if (P->scheme != DECT_SCHEME_UDM_PCG || P->init != DECT_INIT_PCG)
            DECT_FAIL(DECT_EUNSUPPORTED, "dect_admm_create: float64 storage runs the UDM-PCG scheme from the "
                                         "DECT_INIT_PCG start only");
        for (int b = 0; b < B; ++b)
            if (geoms[b] && (geoms[b]->desc.nx > 1024 || geoms[b]->desc.ny > 1024))
                DECT_FAIL(DECT_EUNSUPPORTED, "dect_admm_create: float64 storage supports images up to 1024 x 1024");
    }
    if (P->scheme != DECT_SCHEME_UDM_PCG && P->scheme != DECT_SCHEME_LM_CG)
        DECT_FAIL(DECT_EINVAL, "dect_admm_create: scheme must be DECT_SCHEME_UDM_PCG or DECT_SCHEME_LM_CG");
    if (P->precondition != DECT_PRECOND_NONE && P->precondition != DECT_PRECOND_CIRCULANT &&
        P->precondition != DECT_PRECOND_RAMP)
        DECT_FAIL(DECT_EINVAL, "dect_admm_create: precondition must be DECT_PRECOND_NONE, CIRCULANT or RAMP");
    if (P->scheme == DECT_SCHEME_LM_CG && P->storage != DECT_STORE_F32)
        DECT_FAIL(DECT_EUNSUPPORTED, "dect_admm_create: the LM x CG scheme runs with float32 storage only");
    if (P->bp_view_groups < -1 || P->bp_view_groups > 16)
        DECT_FAIL(DECT_EINVAL, "dect_admm_create: bp_view_groups must be in [-1, 16]");
    if (P->bp_tile != 0 && P->bp_tile != 32 && P->bp_tile != 64)
        DECT_FAIL(DECT_EINVAL, "dect_admm_create: bp_tile must be 0 (autotuned), 32 or 64");
    if (P->bp_cluster < -1 || P->bp_cluster > 1)
        DECT_FAIL(DECT_EINVAL, "dect_admm_create: bp_cluster must be -1 (off), 0 (autotuned) or 1 (on)");
    if (P->bp_slices < 0 || P->bp_slices > 2)
        DECT_FAIL(DECT_EINVAL, "dect_admm_create: bp_slices must be 0 (autotuned), 1 or 2");
    if (P->bp_cluster == 1 && P->bp_slices == 2)
        DECT_FAIL(DECT_EINVAL, "dect_admm_create: bp_cluster = 1 (the cluster form takes one slice per CTA) "
                               "excludes bp_slices = 2");
    if (P->bp_reduce < -1 || P->bp_reduce > 1)
        DECT_FAIL(DECT_EINVAL, "dect_admm_create: bp_reduce must be -1 (off), 0 (default: on) or 1 (on)");
    if (P->proj_views != 0 && P->proj_views != 2 && P->proj_views != 4 && P->proj_views != 8)
        DECT_FAIL(DECT_EINVAL, "dect_admm_create: proj_views must be 0 (autotuned), 2, 4 or 8");
    if (P->init != DECT_INIT_PCG && P->init != DECT_INIT_CDM_FBP)
        DECT_FAIL(DECT_EINVAL, "dect_admm_create: init must be DECT_INIT_PCG or DECT_INIT_CDM_FBP");
    if (P->init == DECT_INIT_CDM_FBP)
        for (int b = 0; b < B; ++b) {
            if (!geoms[b]) break;  // reported below
            const auto& gd = geoms[b]->desc;
            if (gd.kind == DECT_FAN_FLAT ? !span_is(gd.angle_span_rad, 2.0 * M_PI)
                                         : !(span_is(gd.angle_span_rad, M_PI) || span_is(gd.angle_span_rad, 2.0 * M_PI)))
                DECT_FAIL(DECT_EUNSUPPORTED, "dect_admm_create: the CDM-FBP start needs full scans (FBP)");
        }
    if (P->m_udm < 1 || P->n_pcg < 1 || P->m_udm > 64 || P->n_pcg > 64)
        DECT_FAIL(DECT_EINVAL, "dect_admm_create: m_udm and n_pcg must be in [1, 64]");
    if (P->init_udm_iters < 0 || P->init_pcg_iters < 1 || P->init_udm_iters > 1000 || P->init_pcg_iters > 1000)
        DECT_FAIL(DECT_EINVAL, "dect_admm_create: init iterations out of range");
    if (!(P->rho0_c > 0) || !(P->rho0_p > 0) || !(P->lambda_c >= 0) || !(P->lambda_p >= 0) || !(P->rho_mu >= 1) ||
        !(P->rho_tau >= 1) || !(P->lm_mu0 > 0) || !std::isfinite(P->kappa) || !std::isfinite(P->rho0_c) ||
        !std::isfinite(P->rho0_p) || !std::isfinite(P->lambda_c) || !std::isfinite(P->lambda_p))
        DECT_FAIL(DECT_EINVAL, "dect_admm_create: invalid parameter value");
    for (int b = 0; b < B; ++b) {
        if (!geoms[b]) DECT_FAIL(DECT_EINVAL, "dect_admm_create: null geometry");
        if (geoms[b]->desc.nx > 2048 || geoms[b]->desc.ny > 2048)
            DECT_FAIL(DECT_EUNSUPPORTED, "dect_admm_create: the solver supports images up to 2048 x 2048");
    }
    cudaError_t fe = fft_init_attributes();
    if (fe != cudaSuccess) DECT_FAIL(DECT_ECUDA, std::string("dect_admm_create: ") + cudaGetErrorString(fe));

    dect_admm* A = new dect_admm();
    A->B = B;
    A->prec = P->storage;
    A->spec = spec;
    A->P = *P;
    A->geoms.assign(geoms, geoms + B);
    A->has_x0.assign(B, 0);
    A->has_truth.assign(B, 0);
    A->has_data.assign(B, 0);
    for (auto* m : {&A->rays, &A->pix, &A->tx, &A->ty, &A->rows, &A->cols, &A->sweep, &A->cols64, &A->ptile,
                    &A->prows, &A->pcols})
        m->h.assign(1, 0);
    std::vector<int> tune;  // candidate CTA groups per tile when autotuning (first = the occupancy choice)
    std::vector<int> tune_tiles;  // candidate tile sides when autotuning
    {
        cudaError_t ae = sweep_init_attributes();
        if (ae != cudaSuccess) DECT_FAIL(DECT_ECUDA, std::string("dect_admm_create: ") + cudaGetErrorString(ae));
        const int tile0 = P->bp_tile ? P->bp_tile : kSweepTileDefault;
        if (P->bp_tile) tune_tiles.push_back(P->bp_tile);
        else tune_tiles = {64, 32};
        int total = 0;
        int64_t pix = 0;
        for (int b = 0; b < B; ++b) {
            total += sweep_tiles(geoms[b]->desc.nx, geoms[b]->desc.ny, tile0);
            pix += geoms[b]->n_pix();
        }
        A->sweep_tile = tile0;
        A->sweep_reduce = P->bp_reduce >= 0;
        for (int b = 0; b < B; ++b) A->n_tile_count += sweep_tiles(geoms[b]->desc.nx, geoms[b]->desc.ny, 32);
        if (P->bp_cluster == 0) A->cluster_cands = {0, 1};
        else A->cluster_cands = {P->bp_cluster > 0 ? 1 : 0};
        // pairs of consecutive slices of one geometry for the two-slice sweep (UDM-PCG only: the comparison
        // scheme backprojects one basis with its own weights)
        bool pairs = false;
        for (int b = 0; b < B; ++b) {
            if (!A->sgroups.empty() && A->sgroups.back().y < 0 &&
                same_geometry(geoms[A->sgroups.back().x]->desc, geoms[b]->desc)) {
                A->sgroups.back().y = b;
                pairs = true;
            } else {
                A->sgroups.push_back(make_int4(b, -1, -1, -1));
            }
        }
        const bool sg_ok = pairs && P->scheme == DECT_SCHEME_UDM_PCG && P->storage != DECT_STORE_F64;
        if (P->bp_slices == 2 && sg_ok) A->sg_cands = {2};
        else if (P->bp_slices == 0 && sg_ok && P->bp_cluster != 1) A->sg_cands = {1, 2};
        else A->sg_cands = {1};
        A->sweep_sg = A->sg_cands.size() == 1 ? A->sg_cands[0] : 1;
        if (P->storage == DECT_STORE_F64) {
            A->sweep_C = 1;  // the float64 path has its own backprojector; no sweep, no partial images
        } else if (P->bp_view_groups > 0) {
            A->sweep_C = sweep_ctas_for_groups(P->bp_view_groups);
            tune.push_back(A->sweep_C);  // the tile sides and the cluster form may still be timed at this C
        } else if (P->bp_view_groups < 0) {
            A->sweep_C = sweep_groups(total, tile0);  // occupancy choice, not timed
        } else {
            // candidates whose partial images fit in 1/16 of the free memory (and 4 GiB)
            size_t free_b = 0, total_b = 0;
            cudaMemGetInfo(&free_b, &total_b);
            const double budget = std::min(4.0 * (1 << 30), (double)free_b / 16.0);
            const int first = sweep_groups(total, tile0);
            tune.push_back(first);
            for (int c : {4, 6, 8, 10, 12, 16})
                if (c != first && (double)c * pix * sizeof(float2) <= budget) tune.push_back(c);
            A->sweep_C = *std::max_element(tune.begin(), tune.end());
        }
    }
    int64_t max_np = 0, max_nr = 0;
    for (int b = 0; b < B; ++b) {
        const dect_geom* g = geoms[b];
        SliceDesc sd{};
        sd.g = g->dev();
        // slices with the same geometry (every slice of one scan) read one shared ray table: the tables of
        // identical descriptors are identical, and sharing keeps one copy in L2 for the whole batch
        for (int b2 = 0; b2 < b; ++b2)
            if (same_geometry(geoms[b2]->desc, g->desc)) {
                sd.g.rays = geoms[b2]->rays;
                sd.g.views = geoms[b2]->views;
                break;
            }
        const int nx = g->desc.nx, ny = g->desc.ny;
        const int64_t np = g->n_pix(), nr = g->n_rays();
        sd.img_off = A->n_img;
        sd.sino_off = A->n_sino;
        sd.tx_off = A->n_tx;
        sd.ty_off = A->n_ty;
        sd.px = pad_pow2(nx);
        sd.py = pad_pow2(ny);
        sd.lpx = ilog2(sd.px);
        sd.lpy = ilog2(sd.py);
        sd.fft_off = A->n_fft;
        sd.h_off = A->n_h;
        A->n_img += np;
        A->n_sino += nr;
        A->n_tx += (int64_t)nx * (ny + 3);
        A->n_ty += (int64_t)ny * (nx + 3);
        A->n_fft += (int64_t)sd.px * sd.py;
        A->n_h += (int64_t)sd.px * sd.py;
        A->max_px = std::max(A->max_px, sd.px);
        A->max_py = std::max(A->max_py, sd.py);
        A->min_px = std::min(A->min_px, sd.px);
        A->min_py = std::min(A->min_py, sd.py);
        max_np = std::max(max_np, np);
        max_nr = std::max(max_nr, nr);
        A->hs.push_back(sd);
        A->rays.h.push_back(A->rays.h.back() + (int)((nr + kRaysPerBlock - 1) / kRaysPerBlock));

        A->pix.h.push_back(A->pix.h.back() + (int)((np + 255) / 256));
        A->tx.h.push_back(A->tx.h.back() + texture_x_blocks(nx, ny));
        A->ty.h.push_back(A->ty.h.back() + texture_y_blocks(nx, ny));

        A->rows.h.push_back(A->rows.h.back() + ny);
        const int C = precond_cols_per_block(sd.py);
        A->cols.h.push_back(A->cols.h.back() + (sd.px + C - 1) / C);
        const int pr = precond_rows_per_block(sd.px), pc = precond_apply_cols_per_block(sd.py);
        A->prows.h.push_back(A->prows.h.back() + (ny + pr - 1) / pr);
        A->pcols.h.push_back(A->pcols.h.back() + (sd.px + pc - 1) / pc);
        A->cols64.h.push_back(A->cols64.h.back() + sd.px);
    }
    A->n_stage = std::max(4 * max_nr + 4 * max_np, (int64_t)16);
    sweep_prefix(A, A->sweep_C, A->sweep_tile, A->sweep_sg, A->sweep.h);
    // projector groups: a slice joins the previous group when that has room and the same geometry
    std::vector<int4> groups;
    std::vector<int> gsize;
    for (int b = 0; b < B; ++b) {
        if (!groups.empty() && gsize.back() < proj_group_size() &&
            same_geometry(geoms[groups.back().x]->desc, geoms[b]->desc)) {
            int* slot = &groups.back().x;
            slot[gsize.back()++] = b;
        } else {
            groups.push_back(make_int4(b, -1, -1, -1));
            gsize.push_back(1);
        }
    }
    A->n_groups = (int)groups.size();
    for (const int4& gr : groups)
        A->group_shape.push_back(make_int2(geoms[gr.x]->desc.n_views, geoms[gr.x]->desc.n_bins));
    A->proj_views = P->proj_views ? P->proj_views : proj_default_views();
    ptile_prefix(A, A->proj_views, A->ptile.h);

#define ALLOC(ptr, n)                                                      \
    do {                                                                   \
        cudaError_t e_ = dalloc(&(ptr), (size_t)(n));                      \
        if (e_ != cudaSuccess) {                                           \
            dect::set_error(std::string("dect_admm_create: ") + cudaGetErrorString(e_)); \
            free_admm(A);                                                  \
            return DECT_ENOMEM;                                            \
        }                                                                  \
    } while (0)
    ALLOC(A->ds, B);
    ALLOC(A->truth, A->n_img);
    ALLOC(A->meas, A->n_sino);
    ALLOC(A->status, A->n_sino);
    ALLOC(A->stage, A->n_stage);
    ALLOC(A->sc, B);
    ALLOC(A->d_has_x0, B);
    if (A->prec == PREC_F64) {
        F64Vecs& v = A->v64;
        for (double** pp : {&v.x, &v.r, &v.s, &v.p, &v.Ap, &v.z, &v.uz, &v.x0, &v.RTs}) ALLOC(*pp, 2 * A->n_img);
        for (double** pp : {&v.y, &v.uy}) ALLOC(*pp, 4 * A->n_img);
        for (double** pp : {&v.Rx, &v.a, &v.ua, &v.q}) ALLOC(*pp, 2 * A->n_sino);
        ALLOC(v.mu, A->n_sino);
        ALLOC(v.H, A->n_h);
        ALLOC(v.Hn, A->n_h);
        ALLOC(v.Z, A->n_fft);
        for (int b = 0; b < B; ++b) {
            const dect_status ts = geom_table_f64(geoms[b]);
            if (ts != DECT_OK) {
                free_admm(A);
                return ts;
            }
            A->rays64.push_back(geoms[b]->rays64);
        }
    } else {
        for (float2** pp : {&A->x, &A->r, &A->s, &A->p, &A->Ap, &A->z, &A->uz, &A->x0}) ALLOC(*pp, A->n_img);
        for (void** pp : {&A->Rx, &A->a, &A->ua, &A->q}) ALLOC(*(char**)pp, A->n_sino * sino_bytes(A->prec));
        ALLOC(A->y, A->n_img);
        ALLOC(A->uy, A->n_img);
        ALLOC(*(char**)&A->txb, A->n_tx * texel_bytes(A->prec));
        ALLOC(*(char**)&A->tyb, A->n_ty * texel_bytes(A->prec));
        ALLOC(A->mu, A->n_sino);
        ALLOC(A->Z, A->n_fft);
        ALLOC(A->H, A->n_h);
        ALLOC(A->Hn, A->n_h);
        ALLOC(A->Hp, A->n_h);
        ALLOC(A->Hnp, A->n_h);
    }
    if (P->scheme == DECT_SCHEME_LM_CG) {
        ALLOC(A->ls, B);
        ALLOC(A->lm_scale, B);
        for (float** pp : {&A->lm_d, &A->lm_r, &A->lm_p, &A->lm_Ap}) ALLOC(*pp, A->n_img);
        for (float** pp : {&A->lm_e, &A->lm_g, &A->lm_q, &A->lm_Rd}) ALLOC(*pp, A->n_sino);
        ALLOC(A->lm_s0, A->n_sino);
        ALLOC(A->tx1, A->n_tx);
        ALLOC(A->ty1, A->n_ty);
    }
#undef ALLOC
    const int np_blk = A->pix.h.back(), nr_blk = A->rays.h.back();
    cudaError_t e = dalloc(&A->part_udm, 4 * (size_t)nr_blk);
    if (e == cudaSuccess) e = dalloc(&A->part_img, 4 * (size_t)np_blk);
    if (e == cudaSuccess) e = dalloc(&A->part_xi, 4 * (size_t)np_blk);
    if (e == cudaSuccess) e = dalloc(&A->part_rs, 2 * (size_t)A->rows.h.back());
    if (e == cudaSuccess) e = dalloc(&A->part_pap, 2 * (size_t)A->pix.h.back());
    if (e == cudaSuccess) e = dalloc(&A->part_obj_rays, (size_t)nr_blk);
    if (e == cudaSuccess) e = dalloc(&A->part_obj_pix, (size_t)np_blk);
    if (e == cudaSuccess && A->prec != PREC_F64) e = dalloc(&A->bp_partial, (size_t)A->sweep_C * A->n_img);
    if (e == cudaSuccess && A->prec != PREC_F64) e = dalloc(&A->tile_count, (size_t)A->n_tile_count);
    if (e == cudaSuccess && A->prec != PREC_F64) e = cudaMemset(A->tile_count, 0, sizeof(int) * A->n_tile_count);
    // the sweep map holds one entry per unit (slice, or pair of slices of one geometry) plus one; the
    // autotuner's cluster-form trials use the one-slice layout whatever the slices per CTA, so it is
    // sized for B units
    for (MapBuf* m : {&A->rays, &A->pix, &A->tx, &A->ty, &A->rows, &A->cols, &A->sweep, &A->cols64, &A->ptile,
                      &A->prows, &A->pcols})
        if (e == cudaSuccess) e = upload_map(*m, m == &A->sweep ? (size_t)B + 1 : 0);
    if (e == cudaSuccess) e = dalloc(&A->d_groups, groups.size());
    if (e == cudaSuccess) e = dalloc(&A->d_sgroups, A->sgroups.size());
    if (e == cudaSuccess)
        e = cudaMemcpy(A->d_sgroups, A->sgroups.data(), sizeof(int4) * A->sgroups.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(A->d_groups, groups.data(), sizeof(int4) * groups.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(A->ds, A->hs.data(), sizeof(SliceDesc) * B, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(A->truth, 0, sizeof(float2) * A->n_img);
    if (e == cudaSuccess) e = cudaMemset(A->status, 0, A->n_sino);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&A->cap, cudaStreamNonBlocking);
    if (e == cudaSuccess && A->prec != PREC_F64) {
        A->tw = fft_twiddles();
        if (!A->tw) e = cudaErrorMemoryAllocation;
    }
    if (e != cudaSuccess) {
        dect::set_error(std::string("dect_admm_create: ") + cudaGetErrorString(e));
        free_admm(A);
        return e == cudaErrorMemoryAllocation ? DECT_ENOMEM : DECT_ECUDA;
    }
    if (A->prec != PREC_F64 && !tune.empty() &&
        (tune.size() > 1 || tune_tiles.size() > 1 || A->sg_cands.size() > 1 ||
         (A->cluster_cands.size() > 1 && tune[0] >= 2)))
        e = autotune_sweep(A, tune, tune_tiles);
    else if (A->prec != PREC_F64)
        A->sweep_cluster = P->bp_cluster > 0 && A->sweep_sg == 1 && A->sweep_C >= 2 && A->sweep_C <= 16;
    if (e != cudaSuccess) {
        dect::set_error(std::string("dect_admm_create (backprojector autotuning): ") + cudaGetErrorString(e));
        free_admm(A);
        return e == cudaErrorMemoryAllocation ? DECT_ENOMEM : DECT_ECUDA;
    }
    if (A->prec != PREC_F64 && P->proj_views == 0) {
        e = autotune_projector(A);
        if (e != cudaSuccess) {
            dect::set_error(std::string("dect_admm_create (projector autotuning): ") + cudaGetErrorString(e));
            free_admm(A);
            return DECT_ECUDA;
        }
    }
    A->sweep_groups_in_use = A->sweep_C * sweep_groups_per_cta();
    if (P->scheme == DECT_SCHEME_LM_CG) {
        // the comparison scheme has no a-block: its residual slots stay zero for the rho update
        e = cudaMemset(A->part_udm, 0, sizeof(double) * 4 * (size_t)A->rays.h.back());
        if (e == cudaSuccess) e = dalloc(&A->part_lm_pix, (size_t)A->pix.h.back());
        if (e == cudaSuccess) e = dalloc(&A->part_lm_ray, (size_t)A->rays.h.back());
        if (e == cudaSuccess) e = dalloc(&A->bp_partial1, (size_t)A->bp_slots() * A->n_img);
        if (e != cudaSuccess) {
            dect::set_error(std::string("dect_admm_create: ") + cudaGetErrorString(e));
            free_admm(A);
            return e == cudaErrorMemoryAllocation ? DECT_ENOMEM : DECT_ECUDA;
        }
    }
    dect_status s = compute_responses(A);
    if (s != DECT_OK) {
        free_admm(A);
        return s;
    }
    *out = A;
    return DECT_OK;
}

extern "C" void dect_admm_destroy(dect_admm* A) {
    if (!A) return;
    cudaDeviceSynchronize();
    free_admm(A);
}

static dect_status check_slice(const dect_admm* A, int32_t b) {
    if (!A) DECT_FAIL(DECT_EINVAL, "dect_admm: null handle");
    if (b < 0 || b >= A->B) DECT_FAIL(DECT_EINVAL, "dect_admm: slice index out of range");
    return DECT_OK;
}

extern "C" dect_status dect_admm_set_data(dect_admm* A, int32_t b, const float* m_h, const float* m_l,
                                          const float* w_h, const float* w_l, const float* x0, void* stream) {
    clear_stale_error();
    dect_status cs = check_slice(A, b);
    if (cs != DECT_OK) return cs;
    if (!m_h || !m_l || !w_h || !w_l) DECT_FAIL(DECT_EINVAL, "dect_admm_set_data: null measurement array");
    cudaStream_t st = as_stream(stream);
    const SliceDesc& sd = A->hs[b];
    const int64_t nr = (int64_t)sd.g.nv * sd.g.nb, np = (int64_t)sd.g.nx * sd.g.ny;
    const float* src[4] = {m_h, m_l, w_h, w_l};
    for (int k = 0; k < 4; ++k)
        CUDA_TRY(cudaMemcpyAsync(A->stage + k * nr, src[k], sizeof(float) * nr, cudaMemcpyDefault, st));
    launch_pack_meas(A->stage, nr, A->meas + sd.sino_off, st);
    if (x0) {
        CUDA_TRY(cudaMemcpyAsync(A->stage + 4 * nr, x0, sizeof(float) * 2 * np, cudaMemcpyDefault, st));
        if (A->prec == PREC_F64)
            launch64_from_f32(A->stage + 4 * nr, np, A->v64.x0 + 2 * sd.img_off, st);
        else
            launch_interleave(A->stage + 4 * nr, np, A->x0 + sd.img_off, st);
    }
    CUDA_TRY(cudaGetLastError());
    A->has_x0[b] = x0 ? 1 : 0;
    A->has_data[b] = 1;
    A->initialized = false;
    return DECT_OK;
}

extern "C" dect_status dect_admm_set_truth(dect_admm* A, int32_t b, const float* truth, void* stream) {
    clear_stale_error();
    dect_status cs = check_slice(A, b);
    if (cs != DECT_OK) return cs;
    cudaStream_t st = as_stream(stream);
    const SliceDesc& sd = A->hs[b];
    const int64_t np = (int64_t)sd.g.nx * sd.g.ny;
    if (truth) {
        CUDA_TRY(cudaMemcpyAsync(A->stage, truth, sizeof(float) * 2 * np, cudaMemcpyDefault, st));
        launch_interleave(A->stage, np, A->truth + sd.img_off, st);
    } else {
        CUDA_TRY(cudaMemsetAsync(A->truth + sd.img_off, 0, sizeof(float2) * np, st));
    }
    CUDA_TRY(cudaGetLastError());
    A->has_truth[b] = truth ? 1 : 0;
    return DECT_OK;
}

// counters of `iters` replays of the captured iteration (its own counts, taken at capture)
static void count_iterations(dect_admm* A, int iters) {
    A->cR += (int64_t)iters * A->R_per_iter;
    A->cRT += (int64_t)iters * A->RT_per_iter;
    A->cF += (int64_t)iters * A->f_per_iter;
    A->cL += (int64_t)iters * A->launches_per_iter;
}

static dect_status run_iterations(dect_admm* A, int iters, cudaStream_t st) {
    if (A->P.use_graph && !A->gexec) {
        dect_status s = capture_iteration(A, false, &A->gexec);
        if (s != DECT_OK) return s;
    }
    const int k = A->P.objective_every;
    for (int i = 0; i < iters;) {
        // run up to the next iteration whose objective is wanted
        const int n = k > 0 ? std::min(iters - i, (int)(k - A->iters_done % k)) : iters - i;
        if (A->P.use_graph) {
            for (int j = 0; j < n; ++j) CUDA_TRY(cudaGraphLaunch(A->gexec, st));
            count_iterations(A, n);
        } else {
            for (int j = 0; j < n; ++j) enq_iteration(A, st);
        }
        A->iters_done += n;
        i += n;
        if (k > 0 && A->iters_done % k == 0) enq_objective(A, st);
    }
    CUDA_TRY(cudaGetLastError());
    return DECT_OK;
}

extern "C" dect_status dect_admm_profile(dect_admm* A, int32_t iters, void* stream, double* ms, int64_t* launches) {
    clear_stale_error();
    if (!A || !ms || !launches) DECT_FAIL(DECT_EINVAL, "dect_admm_profile: null argument");
    if (iters < 0) DECT_FAIL(DECT_EINVAL, "dect_admm_profile: iters < 0");
    cudaStream_t st = as_stream(stream);
    if (!A->initialized) {
        dect_status s = enq_initialize(A, st);
        if (s != DECT_OK) return s;
    }
    if (A->prof_ev.empty()) {
        A->prof_ev.resize(2 * kMaxProfGroups);
        for (auto& e : A->prof_ev) CUDA_TRY(cudaEventCreate(&e));
    }
    if (!A->pgexec) {
        dect_status s = capture_iteration(A, true, &A->pgexec);
        if (s != DECT_OK) return s;
    }
    A->iters_done += iters;
    for (int i = 0; i < iters; ++i) {
        CUDA_TRY(cudaGraphLaunch(A->pgexec, st));
        CUDA_TRY(cudaStreamSynchronize(st));
        for (int k = 0; k < A->prof_n; ++k) {
            float t = 0.f;
            CUDA_TRY(cudaEventElapsedTime(&t, A->prof_ev[2 * k], A->prof_ev[2 * k + 1]));
            ms[A->prof_phase[k]] += t;
            launches[A->prof_phase[k]] += A->prof_kernels[k];
        }
    }
    count_iterations(A, iters);
    return DECT_OK;
}

extern "C" dect_status dect_admm_step(dect_admm* A, int32_t iters, void* stream) {
    clear_stale_error();
    if (!A) DECT_FAIL(DECT_EINVAL, "dect_admm_step: null handle");
    if (iters < 0) DECT_FAIL(DECT_EINVAL, "dect_admm_step: iters < 0");
    cudaStream_t st = as_stream(stream);
    if (!A->initialized) {
        dect_status s = enq_initialize(A, st);
        if (s != DECT_OK) return s;
    }
    return run_iterations(A, iters, st);
}

extern "C" dect_status dect_reconstruct(dect_admm* A, int32_t iters, void* stream) {
    clear_stale_error();
    if (!A) DECT_FAIL(DECT_EINVAL, "dect_reconstruct: null handle");
    if (iters < 0) DECT_FAIL(DECT_EINVAL, "dect_reconstruct: iters < 0");
    cudaStream_t st = as_stream(stream);
    dect_status s = enq_initialize(A, st);
    if (s != DECT_OK) return s;
    return run_iterations(A, iters, st);
}

extern "C" dect_status dect_admm_get(const dect_admm* A, int32_t b, int32_t which, void* dst, size_t dst_bytes,
                                     void* stream) {
    clear_stale_error();
    dect_status cs = check_slice(A, b);
    if (cs != DECT_OK) return cs;
    if (!dst) DECT_FAIL(DECT_EINVAL, "dect_admm_get: null destination");
    cudaStream_t st = as_stream(stream);
    const SliceDesc& sd = A->hs[b];
    const int64_t np = (int64_t)sd.g.nx * sd.g.ny, nr = (int64_t)sd.g.nv * sd.g.nb;
    size_t need = 0;
    switch (which) {
        case 0: case 6: case 7: need = sizeof(float) * 2 * np; break;
        case 1: case 2: case 3: need = sizeof(float) * 2 * nr; break;
        case 4: case 5: need = sizeof(float) * 4 * np; break;
        case 8: need = sizeof(float) * nr; break;
        case 9: need = sizeof(float) * (size_t)sd.px * sd.py; break;
        default: DECT_FAIL(DECT_EINVAL, "dect_admm_get: unknown array");
    }
    if (A->prec == PREC_F64) {
        // planar float64 arrays: copied as they are
        const F64Vecs& v = A->v64;
        const double* src = nullptr;
        size_t n64 = 0;
        switch (which) {
            case 0: src = v.x + 2 * sd.img_off; n64 = 2 * np; break;
            case 1: src = v.Rx + 2 * sd.sino_off; n64 = 2 * nr; break;
            case 2: src = v.a + 2 * sd.sino_off; n64 = 2 * nr; break;
            case 3: src = v.ua + 2 * sd.sino_off; n64 = 2 * nr; break;
            case 4: src = v.y + 4 * sd.img_off; n64 = 4 * np; break;
            case 5: src = v.uy + 4 * sd.img_off; n64 = 4 * np; break;
            case 6: src = v.z + 2 * sd.img_off; n64 = 2 * np; break;
            case 7: src = v.uz + 2 * sd.img_off; n64 = 2 * np; break;
            case 8: src = v.mu + sd.sino_off; n64 = nr; break;
            default: src = v.H + sd.h_off; n64 = (size_t)sd.px * sd.py; break;
        }
        if (dst_bytes < sizeof(double) * n64) DECT_FAIL(DECT_EINVAL, "dect_admm_get: destination too small");
        CUDA_TRY(cudaMemcpyAsync(dst, src, sizeof(double) * n64, cudaMemcpyDefault, st));
        return DECT_OK;
    }
    if (dst_bytes < need) DECT_FAIL(DECT_EINVAL, "dect_admm_get: destination too small");
    switch (which) {
        case 0: launch_deinterleave2(A->x + sd.img_off, np, A->stage, PREC_F32, st); break;
        case 1: launch_deinterleave2((const char*)A->Rx + sd.sino_off * sino_bytes(A->prec), nr, A->stage, A->prec, st); break;
        case 2: launch_deinterleave2((const char*)A->a + sd.sino_off * sino_bytes(A->prec), nr, A->stage, A->prec, st); break;
        case 3: launch_deinterleave2((const char*)A->ua + sd.sino_off * sino_bytes(A->prec), nr, A->stage, A->prec, st); break;
        case 4: launch_deinterleave4(A->y + sd.img_off, np, A->stage, st); break;
        case 5: launch_deinterleave4(A->uy + sd.img_off, np, A->stage, st); break;
        case 6: launch_deinterleave2(A->z + sd.img_off, np, A->stage, PREC_F32, st); break;
        case 7: launch_deinterleave2(A->uz + sd.img_off, np, A->stage, PREC_F32, st); break;
        default: break;
    }
    if (which == 8)
        CUDA_TRY(cudaMemcpyAsync(dst, A->mu + sd.sino_off, need, cudaMemcpyDefault, st));
    else if (which == 9)
        CUDA_TRY(cudaMemcpyAsync(dst, A->H + sd.h_off, need, cudaMemcpyDefault, st));
    else
        CUDA_TRY(cudaMemcpyAsync(dst, A->stage, need, cudaMemcpyDefault, st));
    CUDA_TRY(cudaGetLastError());
    return DECT_OK;
}

// ---- checkpoint / resume ----------------------------------------------------------------------

namespace {
struct Segment {
    void* p;
    size_t bytes;
};

// the parameters that shape an iteration's arithmetic (a solver resumes only under the same ones)
struct CkptParams {
    double lambda_c, lambda_p, rho0_c, rho0_p, rho_mu, rho_tau, lm_mu0, kappa;
    int32_t m_udm, n_pcg, init_udm_iters, init_pcg_iters, precondition, init, udm_f64, view_groups;
};

struct CkptHeader {
    char magic[8];
    int32_t version, B, storage, scheme, initialized, n_segments;
    int64_t n_img, n_sino, cR, cRT, cF, cL, iters_done;
    CkptParams params;
};

constexpr char kCkptMagic[8] = {'D', 'E', 'C', 'T', 'C', 'K', 'P', 'T'};
constexpr int32_t kCkptVersion = 2;

CkptParams ckpt_params(const dect_admm* A) {
    CkptParams c{};
    const dect_params& P = A->P;
    c.lambda_c = P.lambda_c;
    c.lambda_p = P.lambda_p;
    c.rho0_c = P.rho0_c;
    c.rho0_p = P.rho0_p;
    c.rho_mu = P.rho_mu;
    c.rho_tau = P.rho_tau;
    c.lm_mu0 = P.lm_mu0;
    c.kappa = P.kappa;
    c.m_udm = P.m_udm;
    c.n_pcg = P.n_pcg;
    c.init_udm_iters = P.init_udm_iters;
    c.init_pcg_iters = P.init_pcg_iters;
    c.precondition = P.precondition;
    c.init = P.init;
    c.udm_f64 = P.udm_f64;
    c.view_groups = A->sweep_groups_in_use;  // the view-group count in use fixes the backprojector's sums
    return c;
}

bool same_params(const CkptParams& a, const CkptParams& b) {
    return a.lambda_c == b.lambda_c && a.lambda_p == b.lambda_p && a.rho0_c == b.rho0_c && a.rho0_p == b.rho0_p &&
           a.rho_mu == b.rho_mu && a.rho_tau == b.rho_tau && a.lm_mu0 == b.lm_mu0 && a.kappa == b.kappa &&
           a.m_udm == b.m_udm && a.n_pcg == b.n_pcg && a.init_udm_iters == b.init_udm_iters &&
           a.init_pcg_iters == b.init_pcg_iters && a.precondition == b.precondition && a.init == b.init &&
           a.udm_f64 == b.udm_f64 && a.view_groups == b.view_groups;
}
}  // namespace

// The device arrays that carry state from one iteration to the next (and the data), with the byte
// counts of their allocations in dect_admm_create.
static std::vector<Segment> state_segments(const dect_admm* A) {
    std::vector<Segment> v;
    auto add = [&](const void* p, size_t bytes) {
        if (p && bytes) v.push_back(Segment{const_cast<void*>(p), bytes});
    };
    const size_t ni = (size_t)A->n_img, ns = (size_t)A->n_sino, B = (size_t)A->B;
    if (A->prec == PREC_F64) {
        const F64Vecs& f = A->v64;
        for (const double* p : {f.x, f.r, f.s, f.p, f.Ap, f.z, f.uz, f.x0}) add(p, sizeof(double) * 2 * ni);
        for (const double* p : {f.y, f.uy}) add(p, sizeof(double) * 4 * ni);
        for (const double* p : {f.Rx, f.a, f.ua, f.q}) add(p, sizeof(double) * 2 * ns);
        add(f.mu, sizeof(double) * ns);
        add(A->truth, sizeof(float2) * ni);
        add(A->meas, sizeof(float4) * ns);
        add(A->status, sizeof(uint8_t) * ns);
        add(A->sc, sizeof(SliceScalars) * B);
        add(A->d_has_x0, sizeof(int) * B);
        return v;
    }
    for (const float2* p : {A->x, A->r, A->s, A->p, A->Ap, A->z, A->uz, A->x0, A->truth}) add(p, sizeof(float2) * ni);
    for (const void* p : {A->Rx, A->a, A->ua, A->q}) add(p, ns * sino_bytes(A->prec));
    add(A->y, sizeof(float4) * ni);
    add(A->uy, sizeof(float4) * ni);
    add(A->meas, sizeof(float4) * ns);
    add(A->mu, sizeof(float) * ns);
    add(A->status, sizeof(uint8_t) * ns);
    add(A->sc, sizeof(SliceScalars) * B);
    add(A->d_has_x0, sizeof(int) * B);
    if (A->P.scheme == DECT_SCHEME_LM_CG) {
        add(A->ls, sizeof(LmScalars) * B);
        add(A->lm_scale, sizeof(float) * B);
        for (const float* p : {A->lm_d, A->lm_r, A->lm_p, A->lm_Ap}) add(p, sizeof(float) * ni);
        for (const float* p : {A->lm_e, A->lm_g, A->lm_q, A->lm_Rd}) add(p, sizeof(float) * ns);
        add(A->lm_s0, sizeof(float2) * ns);
    }
    return v;
}

// header, then per slice {nx, ny, n_views, n_bins, has_x0, has_truth, has_data}, then the segments
static size_t ckpt_bytes(const dect_admm* A, const std::vector<Segment>& segs) {
    size_t n = sizeof(CkptHeader) + sizeof(int32_t) * 7 * (size_t)A->B;
    for (const Segment& g : segs) n += g.bytes;
    return n;
}

extern "C" dect_status dect_admm_state_bytes(const dect_admm* A, size_t* bytes) {
    clear_stale_error();
    if (!A || !bytes) DECT_FAIL(DECT_EINVAL, "dect_admm_state_bytes: null argument");
    *bytes = ckpt_bytes(A, state_segments(A));
    return DECT_OK;
}

extern "C" dect_status dect_admm_save(dect_admm* A, void* dst_host, size_t bytes, void* stream) {
    clear_stale_error();
    if (!A || !dst_host) DECT_FAIL(DECT_EINVAL, "dect_admm_save: null argument");
    const std::vector<Segment> segs = state_segments(A);
    const size_t need = ckpt_bytes(A, segs);
    if (bytes < need) DECT_FAIL(DECT_EINVAL, "dect_admm_save: buffer smaller than dect_admm_state_bytes");
    char* out = (char*)dst_host;
    CkptHeader h{};
    std::memcpy(h.magic, kCkptMagic, sizeof(kCkptMagic));
    h.version = kCkptVersion;
    h.B = A->B;
    h.storage = A->P.storage;
    h.scheme = A->P.scheme;
    h.initialized = A->initialized ? 1 : 0;
    h.n_segments = (int32_t)segs.size();
    h.n_img = A->n_img;
    h.n_sino = A->n_sino;
    h.cR = A->cR;
    h.cRT = A->cRT;
    h.cF = A->cF;
    h.cL = A->cL;
    h.iters_done = A->iters_done;
    h.params = ckpt_params(A);
    std::memcpy(out, &h, sizeof(h));
    size_t off = sizeof(h);
    for (int b = 0; b < A->B; ++b) {
        const GeomDev& g = A->hs[b].g;
        const int32_t rec[7] = {g.nx, g.ny, g.nv, g.nb, A->has_x0[b], A->has_truth[b], A->has_data[b]};
        std::memcpy(out + off, rec, sizeof(rec));
        off += sizeof(rec);
    }
    cudaStream_t st = as_stream(stream);
    for (const Segment& g : segs) {
        CUDA_TRY(cudaMemcpyAsync(out + off, g.p, g.bytes, cudaMemcpyDeviceToHost, st));
        off += g.bytes;
    }
    CUDA_TRY(cudaStreamSynchronize(st));
    return DECT_OK;
}

extern "C" dect_status dect_admm_load(dect_admm* A, const void* src_host, size_t bytes, void* stream) {
    clear_stale_error();
    if (!A || !src_host) DECT_FAIL(DECT_EINVAL, "dect_admm_load: null argument");
    const std::vector<Segment> segs = state_segments(A);
    const size_t need = ckpt_bytes(A, segs);
    const char* in = (const char*)src_host;
    CkptHeader h{};
    if (bytes < sizeof(h)) DECT_FAIL(DECT_EINVAL, "dect_admm_load: image too small");
    std::memcpy(&h, in, sizeof(h));
    if (std::memcmp(h.magic, kCkptMagic, sizeof(kCkptMagic)) != 0 || h.version != kCkptVersion)
        DECT_FAIL(DECT_EINVAL, "dect_admm_load: not a dect solver state image");
    if (h.B != A->B || h.storage != A->P.storage || h.scheme != A->P.scheme || h.n_img != A->n_img ||
        h.n_sino != A->n_sino || h.n_segments != (int32_t)segs.size())
        DECT_FAIL(DECT_EINVAL, "dect_admm_load: the image is of a solver with other slices, storage or scheme");
    if (!same_params(h.params, ckpt_params(A)))
        DECT_FAIL(DECT_EINVAL, "dect_admm_load: the image is of a solver with other iteration parameters (lambda, "
                               "rho, m, n, damping, preconditioner, start or backprojector view groups)");
    if (bytes != need) DECT_FAIL(DECT_EINVAL, "dect_admm_load: image size does not match this solver");
    size_t off = sizeof(h);
    std::vector<int32_t> flags(3 * (size_t)A->B);
    for (int b = 0; b < A->B; ++b) {
        int32_t rec[7];
        std::memcpy(rec, in + off, sizeof(rec));
        off += sizeof(rec);
        const GeomDev& g = A->hs[b].g;
        if (rec[0] != g.nx || rec[1] != g.ny || rec[2] != g.nv || rec[3] != g.nb)
            DECT_FAIL(DECT_EINVAL, "dect_admm_load: slice " + std::to_string(b) + " has another shape");
        for (int k = 0; k < 3; ++k) flags[3 * (size_t)b + k] = rec[4 + k];
    }
    cudaStream_t st = as_stream(stream);
    for (const Segment& g : segs) {
        CUDA_TRY(cudaMemcpyAsync(g.p, in + off, g.bytes, cudaMemcpyHostToDevice, st));
        off += g.bytes;
    }
    CUDA_TRY(cudaStreamSynchronize(st));
    for (int b = 0; b < A->B; ++b) {
        A->has_x0[b] = flags[3 * (size_t)b];
        A->has_truth[b] = flags[3 * (size_t)b + 1];
        A->has_data[b] = flags[3 * (size_t)b + 2];
    }
    A->initialized = h.initialized != 0;
    A->cR = h.cR;
    A->cRT = h.cRT;
    A->cF = h.cF;
    A->cL = h.cL;
    A->iters_done = h.iters_done;
    return DECT_OK;
}

extern "C" dect_status dect_admm_stats(dect_admm* A, int32_t b, dect_stats* out, void* stream) {
    clear_stale_error();
    dect_status cs = check_slice(A, b);
    if (cs != DECT_OK) return cs;
    if (!out) DECT_FAIL(DECT_EINVAL, "dect_admm_stats: null output");
    cudaStream_t st = as_stream(stream);
    if (A->has_truth[b]) {
        if (A->prec == PREC_F64) {
            launch64_xi_partials(A->ds, A->pix.map(A->B), A->pix.total, A->v64.x, A->truth, A->part_xi, st);
            launch_xi_reduce(A->part_xi, A->pix.d, A->sc, A->B, st);
        } else {
            launch_xi(A->ds, A->pix.map(A->B), A->pix.total, A->x, A->truth, A->part_xi, A->sc, A->B, st);
        }
    }
    SliceScalars v{};
    CUDA_TRY(cudaMemcpyAsync(&v, A->sc + b, sizeof(v), cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaStreamSynchronize(st));
    out->iteration = v.iteration;
    for (int c = 0; c < 2; ++c) {
        out->rho[c] = v.rho[c];
        out->r_pri[c] = v.r_pri[c];
        out->r_dual[c] = v.r_dual[c];
        out->xi_db[c] = (A->has_truth[b] && v.xi_den[c] > 0) ? 10.0 * std::log10(v.xi_num[c] / v.xi_den[c]) : NAN;
    }
    out->count_R = A->cR;
    out->count_RT = A->cRT;
    out->count_f = A->cF;
    out->count_launches = A->cL;
    out->bp_view_groups = A->sweep_groups_in_use;
    out->objective = v.objective_iter >= 0 ? v.objective : NAN;
    out->objective_iteration = v.objective_iter;
    out->bp_tile = A->prec == PREC_F64 ? 0 : A->sweep_tile;
    out->bp_cluster = A->sweep_cluster ? 1 : 0;
    out->bp_slices = A->prec == PREC_F64 ? 0 : A->sweep_sg;
    out->bp_reduce = A->bp_parts() == 1 && !A->sweep_cluster && A->sweep_C > 1 ? 1 : 0;
    out->proj_views = A->prec == PREC_F64 ? 0 : A->proj_views;
    return DECT_OK;
}
