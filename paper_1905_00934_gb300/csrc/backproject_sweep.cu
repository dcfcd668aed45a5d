// Column-sweep gathering backprojector R^T of the ADMM solver (Table 1's R^T, with the CG
// epilogues of Eq. 12).
//
// A CTA owns a 32 x 32 pixel tile and a group of views; of its two warps one takes the rays
// sampled once per column (axis 0), the other the rays sampled once per row (axis 1). For each
// view a warp stages its rays that can reach the tile (32 at a time) in shared memory, in bin
// order, and walks them. For an axis-0 ray lane c evaluates the sample at column ti + c with the
// same fixed-point integers as the forward projector and adds (1 - f) w s and f w s to the two rows
// it interpolates between; for an axis-1 ray lane r does the same for row tj + r. Each lane thus
// only touches its own column of the warp's accumulator tile ([row][column] for axis 0,
// [column][row] for axis 1: both free of bank conflicts), every sample is evaluated exactly once,
// and no atomics are needed. The two tiles are added in a fixed order into this CTA's partial
// image, and k_bp_finalize adds the C partials of a pixel in a fixed order and applies the
// epilogue, so results are deterministic for a given C.
//
// Staging turns a ray into {tile-relative position at lane 0, slope, w s}: the position is
// q0 + t0 * slope - (a0 << 30) for the tile's first sampled index t0 and first across index a0,
// an exact integer shift, so a lane's floor and fraction equal those of the forward projector at
// the same sample. The ray loop runs in blocks of kSwUnroll rays (the stage padded with null rays:
// far position, zero weight): positions and weights of a block are computed before its
// accumulator updates, and the next chunk's rays are fetched while the current one is processed.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <mutex>
#include <type_traits>
#include <vector>

#include "bp_epilogue.cuh"
#include "dect_internal.cuh"
#include "prec.cuh"
#include "ray_fixed.cuh"

namespace dect {

constexpr int kSw = 32;           // tile side
constexpr int kSwGroups = 1;      // view groups per CTA
constexpr int kSwWarps = 2 * kSwGroups;  // one warp per view group and ray axis
constexpr int kSwRows = kSw + 2;  // accumulator rows -1 .. 32 (the two halo rows are discarded)
constexpr int kSwUnroll = 8;

// NCH = 2: sinogram S2 pairs {c, p}, float2 accumulators and partial images. NCH = 1: float sinogram,
// float accumulators (half the shared-memory traffic), optionally multiplied per ray by rw[ray] and per
// slice by scale[slice] as the rays are staged (the weighted R^T of a Gauss-Newton operator).
template <class S2, int NCH>
__global__ void __launch_bounds__(32 * kSwWarps) k_bp_sweep(const SliceDesc* __restrict__ dsl, BlockMap map, int C,
                                                            const S2* __restrict__ sino,
                                                            typename std::conditional<NCH == 2, float2, float>::type*
                                                                __restrict__ partial,
                                                            int64_t stride, const float* __restrict__ rw,
                                                            const float* __restrict__ scale) {
    using Acc = typename std::conditional<NCH == 2, float2, float>::type;
    // [warp][across index + 1][lane]: [row][column] for axis 0, [column][row] for axis 1
    __shared__ Acc acc[kSwWarps][kSwRows][kSw];
    __shared__ int4 st_ray[kSwWarps][32];  // {position lo, position hi, slope, w s_c}
    __shared__ float st_wp[kSwWarps][32];  // w s_p
    int local;
    const int s = slice_of(map, blockIdx.x, local);
    const SliceDesc& d = dsl[s];
    const GeomDev& g = d.g;
    const int nx = g.nx, ny = g.ny;
    const int c = local % C, tile = local / C;
    const int tiles_x = (nx + kSw - 1) / kSw;
    const int ti = (tile % tiles_x) * kSw, tj = (tile / tiles_x) * kSw;
    const int w = threadIdx.x / 32, lane = threadIdx.x % 32;
    const bool my_axis = w & 1;
    for (int r = 0; r < kSwRows; ++r) acc[w][r][lane] = Acc{};
    const int G = C * kSwGroups, grp = c * kSwGroups + (w >> 1);
    // rays with a weight at the tile's in-image pixels pass within one pixel of their centres:
    // columns ti .. ie, rows tj .. je, widened by one pixel (the rectangle stays inside the image's
    // one-pixel margin, in front of a fan source)
    const int ie = min(ti + kSw, nx) - 1, je = min(tj + kSw, ny) - 1;
    const float xc = (0.5f * (float)(ti + ie) - g.cx) * g.pix, yc = (0.5f * (float)(tj + je) - g.cy) * g.pix;
    const float hx = (0.5f * (float)(ie - ti) + 1.0f) * g.pix, hy = (0.5f * (float)(je - tj) + 1.0f) * g.pix;
    const S2* sn = sino + d.sino_off;
    const int t0 = my_axis ? tj : ti, a0 = my_axis ? ti : tj;
    const long long a0q = (long long)a0 << 30;

    // chunk cursor: view v, first bin k0 of the chunk, last candidate bin khi of the view
    int v = grp, k0 = 0, khi = -1;
    auto seek = [&](int vv) {
        for (v = vv; v < g.nv; v += G) {
            const float4 V = __ldg(g.views + v);
            const CandRange cr = rect_candidates(g, V.x, V.y, xc, yc, hx, hy);
            if (cr.lo <= cr.hi) {
                k0 = cr.lo;
                khi = cr.hi;
                return;
            }
        }
    };
    seek(grp);
    int4 P = make_int4(0, 0, 0, 0);
    float2 sv = make_float2(0.f, 0.f);
    bool have = false;
    auto fetch = [&]() {
        const int k = k0 + lane;
        have = v < g.nv && k <= khi;
        if (have) {
            const size_t e = (size_t)v * g.nb + k;
            P = __ldg(g.rays + e);
            if constexpr (NCH == 2) {
                sv = ldg2(sn + e);
            } else {
                sv.x = __ldg(sn + e);
                if (rw) sv.x *= __ldg(rw + d.sino_off + e);
            }
        }
    };
    fetch();
    const float sscale = (NCH == 1 && scale) ? __ldg(scale + s) : 1.0f;
    while (v < g.nv) {
        // stage this warp's rays of the fetched chunk, compacted in bin order
        const bool mine = have && ray_axis(P) == my_axis;
        const unsigned mask = __ballot_sync(0xffffffffu, mine);
        const int n = __popc(mask);
        if (mine) {
            const long long q = ray_pos(P, t0) - a0q;
            const float wr = ray_w(P) * sscale;
            const int at = __popc(mask & ((1u << lane) - 1u));
            st_ray[w][at] = make_int4((int)(unsigned)(unsigned long long)q, (int)(q >> 32), P.z, __float_as_int(wr * sv.x));
            st_wp[w][at] = wr * sv.y;
        }
        const int nr = (n + kSwUnroll - 1) / kSwUnroll * kSwUnroll;
        if (lane >= n && lane < nr) {  // null rays pad the stage to a multiple of kSwUnroll
            st_ray[w][lane] = make_int4(0, -1000 << 2, 0, 0);
            st_wp[w][lane] = 0.f;
        }
        // advance the cursor and fetch the next chunk while this one is processed
        k0 += 32;
        if (k0 > khi) seek(v + G);
        fetch();
        __syncwarp();
        for (int r0 = 0; r0 < nr; r0 += kSwUnroll) {
            int hh[kSwUnroll];
            float ff[kSwUnroll], wc[kSwUnroll], wp[kSwUnroll];
#pragma unroll
            for (int u = 0; u < kSwUnroll; ++u) {
                const int4 S = st_ray[w][r0 + u];
                const long long q = ((((long long)S.y) << 32) | (long long)(unsigned)S.x) + (long long)lane * S.z;
                hh[u] = pos_floor(q);
                ff[u] = frac_of(q);
                wc[u] = __int_as_float(S.w);
                wp[u] = st_wp[w][r0 + u];
            }
#pragma unroll
            for (int u = 0; u < kSwUnroll; ++u) {
                // rows h, h+1 with h in [-1, 31] are accumulator rows h+1, h+2 (lanes outside skip)
                if ((unsigned)(hh[u] + 1) < (unsigned)(kSw + 1)) {
                    Acc* a = &acc[w][hh[u] + 1][lane];
                    if constexpr (NCH == 2) {
                        float2 x0 = a[0], x1 = a[kSw];
                        x0.x = fmaf(1.0f - ff[u], wc[u], x0.x);
                        x0.y = fmaf(1.0f - ff[u], wp[u], x0.y);
                        x1.x = fmaf(ff[u], wc[u], x1.x);
                        x1.y = fmaf(ff[u], wp[u], x1.y);
                        a[0] = x0;
                        a[kSw] = x1;
                    } else {
                        a[0] = fmaf(1.0f - ff[u], wc[u], a[0]);
                        a[kSw] = fmaf(ff[u], wc[u], a[kSw]);
                    }
                }
            }
        }
        __syncwarp();  // the stage is rewritten by the next chunk
    }
    __syncthreads();
    for (int px = threadIdx.x; px < kSw * kSw; px += blockDim.x) {
        const int rr = px / kSw, cc = px % kSw;
        const int i = ti + cc, j = tj + rr;
        if (i < nx && j < ny) {
            Acc sum{};
            for (int gi = 0; gi < kSwGroups; ++gi) {
                const Acc a = acc[2 * gi][rr + 1][cc], b = acc[2 * gi + 1][cc + 1][rr];
                if constexpr (NCH == 2) {
                    sum.x += a.x + b.x;
                    sum.y += a.y + b.y;
                } else {
                    sum += a + b;
                }
            }
            partial[c * stride + d.img_off + (size_t)j * nx + i] = sum;
        }
    }
}

// (planar != nullptr: single slice, written as [nch][ny][nx] instead of interleaved into `out`)
template <int MODE>
__global__ void __launch_bounds__(256) k_bp_finalize(const SliceDesc* __restrict__ dsl, BlockMap pix, int C,
                                                     const float2* __restrict__ partial, int64_t stride,
                                                     float2* __restrict__ out, BpEpilogue ep,
                                                     float* __restrict__ planar, int nch) {
    int local;
    const int s = slice_of(pix, blockIdx.x, local);
    const SliceDesc& d = dsl[s];
    const int64_t k = (int64_t)local * 256 + threadIdx.x;
    float dot_c = 0.f, dot_p = 0.f;
    if (k < (int64_t)d.g.nx * d.g.ny) {
        const int j = (int)(k / d.g.nx), i = (int)(k % d.g.nx);
        const int64_t e = d.img_off + k;
        float2 acc = make_float2(0.f, 0.f);
        for (int c = 0; c < C; ++c) {
            const float2 v = __ldg(partial + c * stride + e);
            acc.x += v.x;
            acc.y += v.y;
        }
        bp_pixel_epilogue<MODE>(d, i, j, acc, ep, out, planar, nch, dot_c, dot_p);
    }
    if (MODE == BP_AP || MODE == BP_AP_NOGRAD) bp_block_dots(dot_c, dot_p, ep.partial);
}

int sweep_tiles(int nx, int ny) { return ((nx + kSw - 1) / kSw) * ((ny + kSw - 1) / kSw); }

int sweep_ctas_for_groups(int view_groups) { return (view_groups + kSwGroups - 1) / kSwGroups; }
int sweep_groups_per_cta() { return kSwGroups; }

// CTA groups per tile: the smallest C (up to 8) whose grid of tiles * C blocks fills the resident
// slots best (each CTA holds kSwGroups view groups; C * kSwGroups view groups per tile in total).
static std::mutex g_slots_mu;
static std::vector<int> g_slots;  // resident CTA slots of k_bp_sweep, per device

int sweep_groups(int tiles) {
    int dev = 0;
    cudaGetDevice(&dev);
    std::unique_lock<std::mutex> lk(g_slots_mu);
    if ((int)g_slots.size() <= dev) g_slots.resize(dev + 1, 0);
    if (!g_slots[dev]) {
        int sms = 0, occ = 0;
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        // shared memory (34 KB per CTA) limits residency: ask for the largest carve-out
        cudaFuncSetAttribute(k_bp_sweep<float2, 2>, cudaFuncAttributePreferredSharedMemoryCarveout,
                             cudaSharedmemCarveoutMaxShared);
        cudaFuncSetAttribute(k_bp_sweep<__half2, 2>, cudaFuncAttributePreferredSharedMemoryCarveout,
                             cudaSharedmemCarveoutMaxShared);
        cudaFuncSetAttribute(k_bp_sweep<__nv_bfloat162, 2>, cudaFuncAttributePreferredSharedMemoryCarveout,
                             cudaSharedmemCarveoutMaxShared);
        cudaFuncSetAttribute(k_bp_sweep<float, 1>, cudaFuncAttributePreferredSharedMemoryCarveout,
                             cudaSharedmemCarveoutMaxShared);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_bp_sweep<float2, 2>, 32 * kSwWarps, 0);
        g_slots[dev] = sms * (occ > 0 ? occ : 1);
    }
    const int slots = g_slots[dev];
    lk.unlock();
    int best = 1;
    double best_fill = 0.0;
    for (int C = 1; C <= 8; ++C) {
        const long long blocks = (long long)tiles * C;
        const long long waves = (blocks + slots - 1) / slots;
        const double fill = (double)blocks / (double)(waves * slots);
        if (fill > best_fill + 0.05) {
            best = C;
            best_fill = fill;
        }
    }
    return best;
}

void launch_bp_sweep(const SliceDesc* dsl, const BlockMap& smap, int nsweep, int C, const void* sino,
                     float2* partial, int64_t stride, int prec, cudaStream_t st) {
    if (prec == PREC_F16)
        k_bp_sweep<__half2, 2><<<nsweep, 32 * kSwWarps, 0, st>>>(dsl, smap, C, (const __half2*)sino, partial, stride,
                                                                 nullptr, nullptr);
    else if (prec == PREC_BF16)
        k_bp_sweep<__nv_bfloat162, 2><<<nsweep, 32 * kSwWarps, 0, st>>>(dsl, smap, C, (const __nv_bfloat162*)sino,
                                                                         partial, stride, nullptr, nullptr);
    else
        k_bp_sweep<float2, 2><<<nsweep, 32 * kSwWarps, 0, st>>>(dsl, smap, C, (const float2*)sino, partial, stride,
                                                                nullptr, nullptr);
}

void launch_bp_sweep1(const SliceDesc* dsl, const BlockMap& smap, int nsweep, int C, const float* sino, const float* rw,
                      const float* scale, float* partial, int64_t stride, cudaStream_t st) {
    k_bp_sweep<float, 1><<<nsweep, 32 * kSwWarps, 0, st>>>(dsl, smap, C, sino, partial, stride, rw, scale);
}

template <int MODE>
static void finalize_t(const SliceDesc* dsl, const BlockMap& pix, int npix, int C, const float2* partial,
                       int64_t stride, float2* out, const BpEpilogue& ep, cudaStream_t st) {
    k_bp_finalize<MODE><<<npix, 256, 0, st>>>(dsl, pix, C, partial, stride, out, ep, nullptr, 0);
}

void launch_bp_finalize(int mode, const SliceDesc* dsl, const BlockMap& pix, int npix, int C, const float2* partial,
                        int64_t stride, float2* out, const BpEpilogue& ep, cudaStream_t st) {
    switch (mode) {
        case BP_PLAIN: finalize_t<BP_PLAIN>(dsl, pix, npix, C, partial, stride, out, ep, st); break;
        case BP_R0: finalize_t<BP_R0>(dsl, pix, npix, C, partial, stride, out, ep, st); break;
        case BP_AP: finalize_t<BP_AP>(dsl, pix, npix, C, partial, stride, out, ep, st); break;
        case BP_R0_NOGRAD: finalize_t<BP_R0_NOGRAD>(dsl, pix, npix, C, partial, stride, out, ep, st); break;
        case BP_AP_NOGRAD: finalize_t<BP_AP_NOGRAD>(dsl, pix, npix, C, partial, stride, out, ep, st); break;
        default: break;
    }
}

void backproject_single(const SliceDesc& sd, const SliceDesc* d_dev, const int* maps, int C, const float* sino,
                        int nch, float2* packed, float2* partial, float* out, cudaStream_t st) {
    const int64_t nr = (int64_t)sd.g.nv * sd.g.nb, np = (int64_t)sd.g.nx * sd.g.ny;
    launch_pack_planar(sino, nch, nr, packed, st);
    const BlockMap smap{maps, 1}, pmap{maps + 2, 1};
    k_bp_sweep<float2, 2><<<sweep_tiles(sd.g.nx, sd.g.ny) * C, 32 * kSwWarps, 0, st>>>(d_dev, smap, C, packed,
                                                                                      partial, np, nullptr, nullptr);
    k_bp_finalize<BP_PLAIN><<<(unsigned)((np + 255) / 256), 256, 0, st>>>(d_dev, pmap, C, partial, np, nullptr,
                                                                         BpEpilogue{}, out, nch);
}

}  // namespace dect
