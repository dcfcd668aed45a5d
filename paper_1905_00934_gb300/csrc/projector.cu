// Forward projector R and its exact adjoint R^T (the projection matrix of
// Eq. 2-3; Table 1 counts their applications), for parallel and flat-detector
// fan beams.
//
// Sample positions are 34.30 fixed point. A ray is sampled once per column
// (axis 0) or row (axis 1) at position q(t) = q0 + t * slope (t the column or
// row index), so a position is one exact 32x32+64-bit integer multiply-add and
// stepping is an exact 64-bit add: the integer part is the lower
// interpolation neighbour and the top 23 fraction bits give the
// interpolation weight by a bit-cast, without float rounding or conversions.
// Positions carry ~1e-7 pixel error against the exact geometry (float32
// positions would carry ~3e-5 near |q| = 512).
//
// R: one thread per ray, a warp per view and 32 neighbouring bins stepping
// through the sampled columns (rows) in lock step, a CTA per tile of views x
// bins; Joseph's linear interpolation between the two neighbours; the image is
// read through a pair texture (both neighbours of both bases in one 16-byte load).
//
// R^T: the column-sweep kernel of backproject_sweep.cu evaluates the same
// integers per sample, so <R x, y> = <x, R^T y> holds to float32 summation
// rounding; no atomics, deterministic.
#include <cuda_runtime.h>
#include <math.h>

#include "dect_internal.cuh"
#include "bp_epilogue.cuh"
#include "prec.cuh"
#include "ray_fixed.cuh"
#include "f32x2.cuh"

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
    const long long q0_fx = llrint(q0 * 1073741824.0);        // 34.30
    const int slope_fx = (int)llrint(slope * 1073741824.0);    // 2.30, |slope| <= 1
    const float wf = (float)w;
    rays[r] = make_int4((int)(unsigned)(q0_fx & 0xffffffffll), (int)(q0_fx >> 32), slope_fx,
                        __float_as_int(axis ? -wf : wf));
    if (k == 0) views[v] = make_float4((float)c, (float)s, 0.0f, -1.0f);  // z, w: k_view_axes
}

// Axis layout of each view, from the table's own axis bits: bins [0, s1) take the axis of bin 0, bins
// [s1, s2) the other, bins [s2, nb) that of bin 0 again (a flat fan's ray directions span less than a
// quarter turn, so a view switches axis at most twice). Stored in views[v].z = +-(s1 + 1), negative when
// bin 0 is sampled per row, and views[v].w = s2; w = -1 marks a view with more switches (consumers then
// take every bin for both axes).
__global__ void k_view_axes(int nv, int nb, const int4* __restrict__ rays, float4* __restrict__ views) {
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= nv) return;
    const int4* rv = rays + (size_t)v * nb;
    const bool a0 = rv[0].w < 0;
    int k = 1;
    while (k < nb && (rv[k].w < 0) == a0) ++k;
    const int s1 = k;
    while (k < nb && (rv[k].w < 0) != a0) ++k;
    const int s2 = k;
    while (k < nb && (rv[k].w < 0) == a0) ++k;
    const bool mixed = k < nb;
    views[v].z = a0 ? -(float)(s1 + 1) : (float)(s1 + 1);
    views[v].w = mixed ? -1.0f : (float)s2;
}

cudaError_t build_ray_table(const dect_geom_desc& d, int4* rays, float4* views, cudaStream_t st) {
    const int64_t n = (int64_t)d.n_views * d.n_bins;
    k_ray_table<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(d, rays, views);
    k_view_axes<<<(unsigned)((d.n_views + 127) / 128), 128, 0, st>>>(d.n_views, d.n_bins, rays, views);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------------------------
// pair textures

// image value at (j, i), zero outside; IM = float2 {c, p} or float (single channel)
template <class IM>
__device__ __forceinline__ IM img_at(const IM* __restrict__ img, int nx, int ny, int j, int i) {
    if (j < 0 || j >= ny || i < 0 || i >= nx) return IM{};
    return __ldg(img + (size_t)j * nx + i);
}

// TX[i][jj] from a 32 (jj) x 32 (i) tile; rows jj-2 .. jj+29 staged in shared memory.
template <class TX, class IM = float2>
__global__ void __launch_bounds__(256) k_texture_x(const SliceDesc* __restrict__ dsl, BlockMap map,
                                                   const IM* __restrict__ img, TX* __restrict__ tx) {
    __shared__ IM tile[33][33];
    int local;
    const int s = slice_of(map, blockIdx.x, local);
    const SliceDesc& d = dsl[s];
    const int nx = d.g.nx, ny = d.g.ny;
    const int tiles_i = (nx + 31) / 32;
    const int jt = (local / tiles_i) * 32, it = (local % tiles_i) * 32;
    const IM* im = img + d.img_off;
    // stage rows jt-2 .. jt+30 (33 rows), columns it .. it+31
    for (int e = threadIdx.x; e < 33 * 32; e += blockDim.x) {
        const int rr = e / 32, cc = e % 32;
        tile[rr][cc] = img_at(im, nx, ny, jt - 2 + rr, it + cc);
    }
    __syncthreads();
    TX* out = tx + d.tx_off;
    const int ld = ny + 3;
    for (int e = threadIdx.x; e < 32 * 32; e += blockDim.x) {
        const int ci = e / 32, cj = e % 32;  // consecutive threads walk jj: coalesced stores
        const int i = it + ci, jj = jt + cj;
        if (i < nx && jj < ld) sttex(out + (size_t)i * ld + jj, tile[cj][ci], tile[cj + 1][ci]);
    }
}

// TY[j][ii], one entry per thread.
template <class TX, class IM = float2>
__global__ void __launch_bounds__(256) k_texture_y(const SliceDesc* __restrict__ dsl, BlockMap map,
                                                   const IM* __restrict__ img, TX* __restrict__ ty) {
    int local;
    const int s = slice_of(map, blockIdx.x, local);
    const SliceDesc& d = dsl[s];
    const int nx = d.g.nx, ny = d.g.ny, ld = nx + 3;
    const int64_t e = (int64_t)local * blockDim.x + threadIdx.x;
    if (e >= (int64_t)ny * ld) return;
    const int j = (int)(e / ld), ii = (int)(e % ld);
    const IM* im = img + d.img_off;
    sttex(ty + d.ty_off + e, img_at(im, nx, ny, j, ii - 2), img_at(im, nx, ny, j, ii - 1));
}

static int tx_blocks(int nx, int ny) { return ((nx + 31) / 32) * ((ny + 3 + 31) / 32); }
static int ty_blocks(int nx, int ny) { return (int)(((int64_t)ny * (nx + 3) + 255) / 256); }

// Textures of the batched solver: two maps (TX tiles, TY blocks).
void launch_textures(const SliceDesc* dsl, const BlockMap& mx, int nbx, const BlockMap& my, int nby,
                     const float2* img, void* tx, void* ty, int prec, cudaStream_t st) {
    if (prec == PREC_F16) {
        k_texture_x<TexH><<<nbx, 256, 0, st>>>(dsl, mx, img, (TexH*)tx);
        k_texture_y<TexH><<<nby, 256, 0, st>>>(dsl, my, img, (TexH*)ty);
    } else if (prec == PREC_BF16) {
        k_texture_x<TexB><<<nbx, 256, 0, st>>>(dsl, mx, img, (TexB*)tx);
        k_texture_y<TexB><<<nby, 256, 0, st>>>(dsl, my, img, (TexB*)ty);
    } else {
        k_texture_x<float4><<<nbx, 256, 0, st>>>(dsl, mx, img, (float4*)tx);
        k_texture_y<float4><<<nby, 256, 0, st>>>(dsl, my, img, (float4*)ty);
    }
}

// Single-channel textures (float2 texels {x(lo), x(hi)}) of a float image, for the comparison scheme's
// per-basis projections.
void launch_textures1(const SliceDesc* dsl, const BlockMap& mx, int nbx, const BlockMap& my, int nby,
                      const float* img, float2* tx, float2* ty, cudaStream_t st) {
    k_texture_x<float2, float><<<nbx, 256, 0, st>>>(dsl, mx, img, tx);
    k_texture_y<float2, float><<<nby, 256, 0, st>>>(dsl, my, img, ty);
}

// planar input (1 or 2 channels) -> interleaved float2 image
__global__ void k_pack_planar(const float* __restrict__ in, int nch, int64_t n, float2* __restrict__ out) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    out[e] = make_float2(__ldg(in + e), nch > 1 ? __ldg(in + n + e) : 0.0f);
}

// ---------------------------------------------------------------------------------------------
// forward projector

// Launch shape of the forward projector (compile-time; the defaults are the measured best on GB300):
// samples whose texel loads are issued together per lane, views (warps) per CTA, the CTAs per SM the
// register allocation must allow, slices of one geometry per CTA (1, 2 or 4), and whether the
// single-slice sum's positions advance incrementally or are recomputed from the index at every sample
// (both give the same integers, so the same results; the grouped sum always steps incrementally).
#ifndef DECT_PROJ_BATCH
#define DECT_PROJ_BATCH 8
#endif
#ifndef DECT_PROJ_VIEWS
#define DECT_PROJ_VIEWS 2
#endif
#ifndef DECT_PROJ_MINB
#define DECT_PROJ_MINB 16
#endif
#ifndef DECT_PROJ_GROUP
#define DECT_PROJ_GROUP 2
#endif
#ifndef DECT_PROJ_INCR
#define DECT_PROJ_INCR 0
#endif
constexpr int kProjBatch = DECT_PROJ_BATCH;

// The float estimate of a ray's sample range, trimmed with the exact fixed-point positions at its two
// ends, so every sample in [lo, hi] has its lower neighbour in [-2, n_across] (positions are linear
// in t): the texel index (t, floor + 2) then lies inside the padded row [0, n_across + 2] without a
// per-sample clamp. Trimming only drops samples whose two neighbours are both outside the image.
// An empty range comes back as lo > hi.
__device__ __forceinline__ void trimmed_range(const int4 P, const GeomDev& g, int& lo, int& hi) {
    const bool ax = ray_axis(P);
    const int n_along = ax ? g.ny : g.nx, n_across = ax ? g.nx : g.ny;
    sample_range(P, n_along, n_across, lo, hi);
    const long long step = ray_step(P), q0 = ray_q0(P);
    for (int k = 0; k < 4 && lo <= hi; ++k) {
        const int h = pos_floor(q0 + (long long)lo * step);
        if (h >= -2 && h <= n_across) break;
        ++lo;
    }
    for (int k = 0; k < 4 && hi >= lo; ++k) {
        const int h = pos_floor(q0 + (long long)hi * step);
        if (h >= -2 && h <= n_across) break;
        --hi;
    }
    if (lo <= hi) {
        // the trimming loops stop after 4 steps; re-check so that no sample can index outside its row
        const int h0 = pos_floor(q0 + (long long)lo * step), h1 = pos_floor(q0 + (long long)hi * step);
        if (h0 < -2 || h0 > n_across || h1 < -2 || h1 > n_across) hi = lo - 1;
    }
}

// One sample's interpolated {c, p} from the texel pair {c0, p0, c1, p1} at upper weight f, as a
// packed pair: {fma(f, c1 - c0, c0), fma(f, p1 - p0, p0)}, each element rounded as in scalar code.
__device__ __forceinline__ f32x2 lerp2(float f, const float4 v) {
    const f32x2 lo = pack2(v.x, v.y);
    return fma2(pack2(f, f), sub2(pack2(v.z, v.w), lo), lo);
}

// Sum over a ray's samples of the interpolated {c, p} (unweighted), with the warp stepping in lock
// step: every lane visits the same sampled index t, from the warp's lowest first index to its highest
// last one, so at each step the lanes (neighbouring rays) read neighbouring texels of one texture row
// and their loads coalesce. A lane outside its own [lo, hi] reads texel 0 of its texture, which is
// always zero padding (the pair of rows or columns -2, -1 of column or row 0), and adds an exact zero,
// so each ray's sum takes the same terms in the same order as a walk over its own range alone.
// Every lane of the warp must call this (valid = false for lanes without a ray).
template <class TX>
__device__ __forceinline__ float2 ray_sum_sync(const int4 P, bool valid, const GeomDev& g, const TX* __restrict__ tx,
                                               const TX* __restrict__ ty) {
    const bool ax = ray_axis(P);
    const int n_across = ax ? g.nx : g.ny;
    const TX* __restrict__ tex = ax ? ty : tx;
    const int ld = n_across + 3;
    int lo = 1, hi = 0;
    if (valid) trimmed_range(P, g, lo, hi);
    const bool any = lo <= hi;
    const int t0 = __reduce_min_sync(0xffffffffu, any ? lo : 0x7fffffff);
    const int t1 = __reduce_max_sync(0xffffffffu, any ? hi : -1);
    // {c, p} sums as one packed pair: each element's terms and order are those of two scalar sums
    f32x2 acc = pack2(0.f, 0.f);
    if (t0 > t1) return unpack2(acc);  // no lane of the warp samples the image (warp-uniform)
    // from here 0 <= t0 <= t1 < max(nx, ny): the bounds below cannot overflow
    const long long step = ray_step(P), q0 = ray_q0(P);
    int t = t0;
#if DECT_PROJ_INCR
    // positions and texel rows advance by exact integer steps; a lane samples while (t - lo), modulo 2^32
    // (it wraps through 0 exactly when t reaches lo), is <= hi - lo. A lane without samples starts at
    // 2^31 with len 0: its rel stays in [2^31, 2^31 + 4104) over at most 4096 + 8 steps, never <= 0.
    long long q = q0 + (long long)t0 * step;
    int base = t0 * ld + 2;  // texel (t, floor + 2) is tex[base + floor(q)]
    unsigned rel = any ? (unsigned)(t0 - lo) : 0x80000000u;
    const unsigned len = any ? (unsigned)(hi - lo) : 0u;
    for (; t <= t1 - (kProjBatch - 1); t += kProjBatch) {
        float4 v[kProjBatch];
        float f[kProjBatch];
#pragma unroll
        for (int u = 0; u < kProjBatch; ++u) {
            v[u] = make_float4(0.f, 0.f, 0.f, 0.f);
            if (rel + (unsigned)u <= len) v[u] = ldtex(tex + (base + pos_floor(q)));
            f[u] = frac_of(q);
            q += step;
            base += ld;
        }
        rel += kProjBatch;
#pragma unroll
        for (int u = 0; u < kProjBatch; ++u) acc = add2(acc, lerp2(f[u], v[u]));
    }
#else
    for (; t <= t1 - (kProjBatch - 1); t += kProjBatch) {
        float4 v[kProjBatch];
        float f[kProjBatch];
#pragma unroll
        for (int u = 0; u < kProjBatch; ++u) {
            const int tt = t + u;
            const long long qu = q0 + (long long)tt * step;
            // a lane outside its range reads texel 0, which is zero padding (rows or columns -2 and -1)
            const int idx = (tt >= lo && tt <= hi) ? tt * ld + 2 + pos_floor(qu) : 0;
            v[u] = ldtex(tex + idx);
            f[u] = frac_of(qu);
        }
#pragma unroll
        for (int u = 0; u < kProjBatch; ++u) acc = add2(acc, lerp2(f[u], v[u]));
    }
#endif
    for (; t <= t1; ++t) {
        const long long q1 = q0 + (long long)t * step;
        const float4 v = ldtex(tex + ((t >= lo && t <= hi) ? t * ld + 2 + pos_floor(q1) : 0));
        acc = add2(acc, lerp2(frac_of(q1), v));
    }
    return unpack2(acc);
}

// A CTA takes a tile of V consecutive views x 32 consecutive bins, one warp per view: the rays of
// neighbouring views through the same bins cross nearly the same texels, so the tile's warps share them
// in L1. V = 2, 4 or 8 is timed by the solver at creation (a ray's sum does not depend on its tile, so
// every V gives the same bits); kProjViews is the default and the single-slice projector's.
constexpr int kProjViews = DECT_PROJ_VIEWS;
constexpr int kProjGroup = DECT_PROJ_GROUP;  // slices of one geometry projected by one CTA (<= 4)

__host__ __device__ __forceinline__ int proj_bin_tiles(int nb) { return (nb + 31) / 32; }

int proj_tiles(int nv, int nb, int views) { return ((nv + views - 1) / views) * proj_bin_tiles(nb); }
int proj_default_views() { return kProjViews; }

// (view, bin) of this thread in tile `local` of a slice with nv views and nb bins, V views per tile
template <int V>
__device__ __forceinline__ bool proj_ray(int local, int nv, int nb, int& v, int& k) {
    const int nbt = proj_bin_tiles(nb);
    v = (local / nbt) * V + (int)(threadIdx.x >> 5);
    k = (local % nbt) * 32 + (int)(threadIdx.x & 31);
    return v < nv && k < nb;
}

// The same lock-step sum for the rays of one geometry through up to G slices' images at once (slices
// of one scan share the geometry): positions, ranges and texel indices are formed once per sample and
// only the texel loads and the accumulation are per slice. Each slice's sum takes the same terms in the
// same order as ray_sum_sync on that slice alone. count (<= G) is uniform over the CTA.
template <class TX, int G>
__device__ __forceinline__ void ray_sum_group(const int4 P, bool valid, const GeomDev& g, const TX* const (&txs)[G],
                                              const TX* const (&tys)[G], int count, float2 (&acc)[G]) {
    const bool ax = ray_axis(P);
    const int n_across = ax ? g.nx : g.ny;
    const int ld = n_across + 3;
    int lo = 1, hi = 0;
    if (valid) trimmed_range(P, g, lo, hi);
    const bool any = lo <= hi;
    const int t0 = __reduce_min_sync(0xffffffffu, any ? lo : 0x7fffffff);
    const int t1 = __reduce_max_sync(0xffffffffu, any ? hi : -1);
    f32x2 acc2[G];  // {c, p} sums per slice as packed pairs
#pragma unroll
    for (int k = 0; k < G; ++k) acc2[k] = pack2(0.f, 0.f);
    if (t0 <= t1) {  // some lane of the warp samples the image (warp-uniform)
        // from here 0 <= t0 <= t1 < max(nx, ny): the bounds below cannot overflow
        const long long step = ray_step(P), q0 = ray_q0(P);
        const TX* tex[G];
#pragma unroll
        for (int k = 0; k < G; ++k) tex[k] = ax ? tys[k] : txs[k];
        int t = t0;
        // position and texel row of sample t, stepped exactly: q = q0 + t step, base = t ld + 2
        long long q = q0 + (long long)t0 * step;
        int base = t0 * ld + 2;
        for (; t <= t1 - (kProjBatch - 1); t += kProjBatch) {
            int idx[kProjBatch];
            float f[kProjBatch];
#pragma unroll
            for (int u = 0; u < kProjBatch; ++u) {
                const int tt = t + u;
                idx[u] = (tt >= lo && tt <= hi) ? base + pos_floor(q) : 0;  // texel 0: zero padding
                f[u] = frac_of(q);
                q += step;
                base += ld;
            }
#pragma unroll
            for (int k = 0; k < G; ++k) {
                if (k >= count) break;
                float4 v[kProjBatch];
#pragma unroll
                for (int u = 0; u < kProjBatch; ++u) v[u] = ldtex(tex[k] + idx[u]);
#pragma unroll
                for (int u = 0; u < kProjBatch; ++u) acc2[k] = add2(acc2[k], lerp2(f[u], v[u]));
            }
        }
        for (; t <= t1; ++t, q += step, base += ld) {
            const int i1 = (t >= lo && t <= hi) ? base + pos_floor(q) : 0;
            const float f = frac_of(q);
#pragma unroll
            for (int k = 0; k < G; ++k) {
                if (k >= count) break;
                acc2[k] = add2(acc2[k], lerp2(f, ldtex(tex[k] + i1)));
            }
        }
    }
#pragma unroll
    for (int k = 0; k < G; ++k) acc[k] = unpack2(acc2[k]);
}

// One CTA per (geometry group, tile): group gi holds up to kProjGroup slices of one geometry (their
// indices in groups[gi], -1 past the group's size); the block map counts tiles per group.
// (the register budget allows DECT_PROJ_MINB 64-thread CTAs per SM, the same warps for every V)
template <class S2, class TX, int V>
__global__ void __launch_bounds__(32 * V, DECT_PROJ_MINB * 2 / V) k_project(const SliceDesc* __restrict__ dsl,
                                                                          BlockMap map, const int4* __restrict__ groups,
                                                                          const TX* __restrict__ tx,
                                                                          const TX* __restrict__ ty, S2* __restrict__ out) {
    int local;
    const int gi = slice_of(map, blockIdx.x, local);
    const int4 gs = __ldg(groups + gi);
    const int all[4] = {gs.x, gs.y, gs.z, gs.w};
    int sl[kProjGroup];
#pragma unroll
    for (int q = 0; q < kProjGroup; ++q) sl[q] = all[q];
    const int count = 1 + (gs.y >= 0) + (gs.z >= 0) + (gs.w >= 0);
    const SliceDesc& d = dsl[sl[0]];
    int v, k;
    const bool valid = proj_ray<V>(local, d.g.nv, d.g.nb, v, k);
    const int64_t r = (int64_t)v * d.g.nb + k;
    const int4 P = valid ? __ldg(d.g.rays + r) : make_int4(0, 0, 0, 0);
    const TX* txs[kProjGroup];
    const TX* tys[kProjGroup];
#pragma unroll
    for (int q = 0; q < kProjGroup; ++q) {
        const SliceDesc& dq = dsl[q < count ? sl[q] : sl[0]];
        txs[q] = tx + dq.tx_off;
        tys[q] = ty + dq.ty_off;
    }
    float2 acc[kProjGroup];
    ray_sum_group<TX, kProjGroup>(P, valid, d.g, txs, tys, count, acc);
    const float w = ray_w(P);
    if (!valid) return;
#pragma unroll
    for (int q = 0; q < kProjGroup; ++q)
        if (q < count) st2(out + dsl[sl[q]].sino_off + r, make_float2(w * acc[q].x, w * acc[q].y));
}

__global__ void __launch_bounds__(32 * kProjViews, DECT_PROJ_MINB) k_project_planar(SliceDesc d, const float4* __restrict__ tx,
                                                                    const float4* __restrict__ ty,
                                                                    float* __restrict__ out, int nch) {
    const int64_t n = (int64_t)d.g.nv * d.g.nb;
    int v, k;
    const bool valid = proj_ray<kProjViews>(blockIdx.x, d.g.nv, d.g.nb, v, k);
    const int64_t r = (int64_t)v * d.g.nb + k;
    const int4 P = valid ? __ldg(d.g.rays + r) : make_int4(0, 0, 0, 0);
    const float2 acc = ray_sum_sync(P, valid, d.g, tx, ty);
    const float w = ray_w(P);
    if (!valid) return;
    out[r] = w * acc.x;
    if (nch > 1) out[n + r] = w * acc.y;
}

template <class S2, class TX>
static void project_t(const SliceDesc* dsl, const BlockMap& map, int nblk, const int4* groups, const TX* tx,
                      const TX* ty, S2* out, int views, cudaStream_t st) {
    if (views == 8)
        k_project<S2, TX, 8><<<nblk, 256, 0, st>>>(dsl, map, groups, tx, ty, out);
    else if (views == 4)
        k_project<S2, TX, 4><<<nblk, 128, 0, st>>>(dsl, map, groups, tx, ty, out);
    else
        k_project<S2, TX, 2><<<nblk, 64, 0, st>>>(dsl, map, groups, tx, ty, out);
}

void launch_project(const SliceDesc* dsl, const BlockMap& map, int nblk, const int4* groups, const void* tx,
                    const void* ty, void* out, int prec, int views, cudaStream_t st) {
    if (prec == PREC_F16)
        project_t(dsl, map, nblk, groups, (const TexH*)tx, (const TexH*)ty, (__half2*)out, views, st);
    else if (prec == PREC_BF16)
        project_t(dsl, map, nblk, groups, (const TexB*)tx, (const TexB*)ty, (__nv_bfloat162*)out, views, st);
    else
        project_t(dsl, map, nblk, groups, (const float4*)tx, (const float4*)ty, (float2*)out, views, st);
}

// single channel: float out, float2 texels
void launch_project1(const SliceDesc* dsl, const BlockMap& map, int nblk, const int4* groups, const float2* tx,
                     const float2* ty, float* out, int views, cudaStream_t st) {
    project_t(dsl, map, nblk, groups, tx, ty, out, views, st);
}

int proj_group_size() { return kProjGroup; }

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
// The buffers passed here are the slice's own (already offset), so the descriptor's offsets are
// cleared before the kernels see it.
void project_single(const SliceDesc& sd_in, const float* img, int nch, float2* scratch, float4* tx, float4* ty,
                    float* out, cudaStream_t st) {
    SliceDesc sd = sd_in;
    sd.img_off = sd.sino_off = sd.tx_off = sd.ty_off = sd.fft_off = sd.h_off = 0;
    const int64_t np = (int64_t)sd.g.nx * sd.g.ny;
    k_pack_planar<<<(unsigned)((np + 255) / 256), 256, 0, st>>>(img, nch, np, scratch);
    k_texture_x_single<<<tx_blocks(sd.g.nx, sd.g.ny), 256, 0, st>>>(sd, scratch, tx);
    k_texture_y_single<<<ty_blocks(sd.g.nx, sd.g.ny), 256, 0, st>>>(sd, scratch, ty);
    k_project_planar<<<proj_tiles(sd.g.nv, sd.g.nb, kProjViews), 32 * kProjViews, 0, st>>>(sd, tx, ty, out, nch);
}

void launch_pack_planar(const float* in, int nch, int64_t n, float2* out, cudaStream_t st) {
    k_pack_planar<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(in, nch, n, out);
}

int texture_x_blocks(int nx, int ny) { return tx_blocks(nx, ny); }
int texture_y_blocks(int nx, int ny) { return ty_blocks(nx, ny); }

}  // namespace dect
