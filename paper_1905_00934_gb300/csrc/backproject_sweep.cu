// Column-sweep gathering backprojector R^T of the ADMM solver (Table 1's R^T, with the CG
// epilogues of Eq. 12).
//
// A CTA owns a pixel tile (32 x 32 or 64 x 64, see SweepShape) and a group of views; its warps take
// the rays sampled once per column (axis 0) or once per row (axis 1) over bands of the tile. For each
// view a warp stages its rays that can reach the tile (32 at a time) in shared memory, in bin
// order, and walks them; it fetches only the bins of its own axis (each view's axis layout is
// recorded with the geometry: a view switches axis at most twice). For an axis-0 ray lane c evaluates the sample at column ti + c with the
// same fixed-point integers as the forward projector and adds (1 - f) w s and f w s to the two rows
// it interpolates between; for an axis-1 ray lane r does the same for row tj + r. Each lane thus
// only touches its own column of the warp's accumulator tile ([row][column] for axis 0,
// [column][row] for axis 1: both free of bank conflicts), every sample is evaluated exactly once,
// and no atomics are needed. The two tiles are added in a fixed order into this CTA's partial
// image, and k_bp_finalize adds the C partials of a pixel in a fixed order and applies the
// epilogue, so results are deterministic for a given C. In the reduced form the last of a tile's C
// CTAs to finish (a per-tile arrival counter) forms that same sum while the partials are still in L2,
// writes it to partial image 0 (the finalize pass then reads one image) and drops the L2 lines of the
// other partials it consumed, so they are never written back to DRAM.
//
// Staging turns a ray into {tile-relative position at lane 0, slope, w s}: the position is
// q0 + t0 * slope - (a0 << 30) for the tile's first sampled index t0 and first across index a0,
// an exact integer shift, so a lane's floor and fraction equal those of the forward projector at
// the same sample. The ray loop runs in blocks of kSwUnroll rays (the stage padded with null rays:
// far position, zero weight): positions and weights of a block are computed before its
// accumulator updates, and the next chunk's rays are fetched while the current one is processed.
#include <cooperative_groups.h>
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
#include "f32x2.cuh"

namespace dect {

// A tile is TILE x TILE pixels (TILE = 32 or 64) and its CTA has 2 * TILE / 32 warps: the first
// TILE / 32 take the rays sampled once per column (axis 0), each for a band of 32 columns x TILE
// rows, the others the rays sampled once per row (axis 1), each for a band of TILE columns x 32 rows.
// A taller band leaves fewer lanes idle on rays that clip a corner of it (a CPU model of the 512^2
// fan workload: 72 % of a staged ray's lanes sample the band at 32 rows, 83 % at 64), at the price of
// twice the accumulator per warp. Both shapes evaluate every sample once, in the same order per
// pixel within a view group, and the autotuner of the solver picks one by timing.
#ifndef DECT_SW_UNROLL
#define DECT_SW_UNROLL 8
#endif
constexpr int kSwUnroll = DECT_SW_UNROLL;  // rays per block of the sweep's inner loop (a multiple of 4)
// 4 and 8 give the same bits (both measured); 16 ran as fast but its images drifted from theirs within a
// few iterations, for a reason not found, so it is not allowed.
static_assert(kSwUnroll == 4 || kSwUnroll == 8, "rays per block: 4 or 8");

// Drop the L2 lines that lie wholly inside [lo, hi) without writing them back (discard.global.L2,
// 128-byte lines; their contents become undefined). The caller owns every byte of the range.
__device__ __forceinline__ void discard_l2_range(const void* lo, const void* hi) {
    size_t a = (__cvta_generic_to_global(lo) + 127) & ~(size_t)127;
    const size_t e = __cvta_generic_to_global(hi);
    for (; a + 128 <= e; a += 128) asm volatile("discard.global.L2 [%0], 128;" ::"l"(a) : "memory");
}

template <int TILE>
struct SweepShape {
    static constexpr int kBands = TILE / 32;      // bands per axis
    static constexpr int kWarps = 2 * kBands;     // one warp per band and axis
    static constexpr int kRows = TILE + 2;        // accumulator rows (across index -1 .. TILE; halo discarded)
    static constexpr int kThreads = 32 * kWarps;
};

// shared-memory bytes of a CTA's accumulators (dynamic shared memory), SG slices per CTA
template <int TILE, int NCH, int SG = 1>
constexpr size_t sweep_acc_bytes() {
    return (size_t)SG * SweepShape<TILE>::kWarps * SweepShape<TILE>::kRows * 32 *
           (NCH == 2 ? sizeof(float2) : sizeof(float));
}

// NCH = 2: sinogram S2 pairs {c, p}, float2 accumulators and partial images. NCH = 1: float sinogram,
// float accumulators (half the shared-memory traffic), optionally multiplied per ray by rw[ray] and per
// slice by scale[slice] as the rays are staged (the weighted R^T of a Gauss-Newton operator).
// CLUSTER: the C CTAs of a tile (consecutive blocks) form a thread-block cluster and add their
// accumulators through distributed shared memory, in rank order, into one partial image (image 0);
// the sum per pixel is the one the finalize pass forms from C partial images (0 + p_0 + p_1 + ...),
// so both launch forms give the same bits, and only one image per tile goes through L2 and DRAM.
// SG = 2: a CTA backprojects the same rays into two slices of one geometry (their indices in
// groups[unit], the second -1 if the group has one slice): staging, candidate search and sample
// positions are done once, each slice has its own accumulators, and each slice's pixels receive the
// same contributions in the same order as with SG = 1 (the same bits). NCH = 2, plain form only.
// tile_count != nullptr (plain form): the reduced form. One counter per tile of the launch (block /
// C), zero on entry; the tile's last CTA adds 0 + p_0 + ... + p_{C-1} per pixel, the finalize pass's
// sum, into image 0 and sets the counter back to zero.
template <class S2, int NCH, int TILE, bool CLUSTER = false, int SG = 1>
__global__ void __launch_bounds__(SweepShape<TILE>::kThreads) k_bp_sweep(
    const SliceDesc* __restrict__ dsl, BlockMap map, int C, const int4* __restrict__ groups,
    const S2* __restrict__ sino, typename std::conditional<NCH == 2, float2, float>::type* __restrict__ partial,
    int64_t stride, const float* __restrict__ rw, const float* __restrict__ scale, int* __restrict__ tile_count) {
    static_assert(SG == 1 || (SG == 2 && NCH == 2 && !CLUSTER), "two slices per CTA: two channels, plain form");
    using Acc = typename std::conditional<NCH == 2, float2, float>::type;
    using Sh = SweepShape<TILE>;
    // [slice][warp][across index + 1][lane]: [row][column] for axis 0, [column][row] for axis 1
    extern __shared__ __align__(16) unsigned char sweep_smem[];
    Acc(*acc_all)[Sh::kWarps][Sh::kRows][32] = reinterpret_cast<Acc(*)[Sh::kWarps][Sh::kRows][32]>(sweep_smem);
    Acc(*acc)[Sh::kRows][32] = acc_all[0];
    // SG = 2: one float4 {c, p of the first slice, c, p of the second} per accumulator cell, so a sample's
    // update of both slices is one 16-byte read-modify-write per row (the same bytes as two 8-byte ones)
    float4(*acc4)[Sh::kRows][32] = reinterpret_cast<float4(*)[Sh::kRows][32]>(sweep_smem);
    __shared__ int4 st_ray[Sh::kWarps][32];                 // {position lo, position hi, slope, w s_c}
    __shared__ __align__(16) float st_wp[Sh::kWarps][32];   // w s_p (SG = 1)
    // SG = 2: {w s_c, w s_p, w s_c', w s_p'} of both slices, as two packed pairs for the accumulator update
    __shared__ float4 st_w2[SG == 2 ? Sh::kWarps : 1][32];
    int local;
    const int unit = slice_of(map, blockIdx.x, local);
    int sl[SG];
    int count = 1;
    if constexpr (SG == 1) {
        sl[0] = unit;
    } else {
        const int4 gs = __ldg(groups + unit);
        sl[0] = gs.x;
        sl[1] = gs.y >= 0 ? gs.y : gs.x;
        count = gs.y >= 0 ? 2 : 1;
    }
    const int s = sl[0];
    const SliceDesc& d = dsl[s];
    const GeomDev& g = d.g;
    const int nx = g.nx, ny = g.ny;
    const int c = local % C, tile = local / C;
    const int tiles_x = (nx + TILE - 1) / TILE;
    const int ti = (tile % tiles_x) * TILE, tj = (tile / tiles_x) * TILE;
    const int w = threadIdx.x / 32, lane = threadIdx.x % 32;
    const bool my_axis = w >= Sh::kBands;
    const int band = w % Sh::kBands;
    if constexpr (SG == 2) {
        for (int r = 0; r < Sh::kRows; ++r) acc4[w][r][lane] = make_float4(0.f, 0.f, 0.f, 0.f);
    } else {
        for (int r = 0; r < Sh::kRows; ++r) acc[w][r][lane] = Acc{};
    }
    const int G = C, grp = c;
    // this warp's band: 32 sampled indices from bi (columns for axis 0, rows for axis 1) by the tile's
    // TILE across indices from ba; rays with a weight at its in-image pixels pass within one pixel of
    // their centres, so candidates come from the band's rectangle widened by one pixel (inside the
    // image's one-pixel margin, in front of a fan source)
    const int bi = (my_axis ? tj : ti) + 32 * band, ba = my_axis ? ti : tj;
    const int n_along = my_axis ? ny : nx, n_across = my_axis ? nx : ny;
    const int be = min(bi + 32, n_along) - 1, ae = min(ba + TILE, n_across) - 1;
    const bool empty = bi >= n_along;  // a band past the image's last column / row (ragged tiles)
    const int i0 = my_axis ? ba : bi, i1 = my_axis ? ae : be, j0 = my_axis ? bi : ba, j1 = my_axis ? be : ae;
    const float xc = (0.5f * (float)(i0 + i1) - g.cx) * g.pix, yc = (0.5f * (float)(j0 + j1) - g.cy) * g.pix;
    const float hx = (0.5f * (float)(i1 - i0) + 1.0f) * g.pix, hy = (0.5f * (float)(j1 - j0) + 1.0f) * g.pix;
    const S2* sn = sino + d.sino_off;
    const S2* sn1 = sino + dsl[sl[SG - 1]].sino_off;  // the second slice's sinogram (SG = 2)
    const long long a0q = (long long)ba << 30;

    // chunk cursor: view v, first bin k0 of the chunk, last bin khi of the current candidate interval,
    // [k2, k2hi] a second interval of the view still to come. A view's candidates are the bins whose
    // rays can reach the band, restricted to the bins of this warp's axis (the view's axis layout), so
    // the warp fetches only rays it stages; the rays keep their bin order.
    int v = empty ? g.nv : grp, k0 = 0, khi = -1, k2 = 1, k2hi = 0;
    auto seek = [&](int vv) {
        for (v = vv; v < g.nv; v += G) {
            const float4 V = __ldg(g.views + v);
            const CandRange cr = rect_candidates(g, V.x, V.y, xc, yc, hx, hy);
            if (cr.lo > cr.hi) continue;
            int a1 = 0, b1 = g.nb - 1, a2 = 1, b2 = 0;  // a mixed layout: every bin, one interval
            if (V.w >= 0.f && fabsf(V.z) >= 1.f) {
                const bool ax0 = V.z < 0.f;
                const int s1 = (int)fabsf(V.z) - 1, s2 = (int)V.w;
                if (ax0 == my_axis) {
                    b1 = s1 - 1;
                    a2 = s2;
                    b2 = g.nb - 1;
                } else {
                    a1 = s1;
                    b1 = s2 - 1;
                }
            }
            const int l1 = max(cr.lo, a1), h1 = min(cr.hi, b1), l2 = max(cr.lo, a2), h2 = min(cr.hi, b2);
            if (l1 <= h1) {
                k0 = l1;
                khi = h1;
                k2 = l2;
                k2hi = h2;
                return;
            }
            if (l2 <= h2) {
                k0 = l2;
                khi = h2;
                k2 = 1;
                k2hi = 0;
                return;
            }
        }
    };
    if (!empty) seek(grp);
    int4 P = make_int4(0, 0, 0, 0);
    float2 sv = make_float2(0.f, 0.f), sv1 = make_float2(0.f, 0.f);
    bool have = false;
    auto fetch = [&]() {
        const int k = k0 + lane;
        have = v < g.nv && k <= khi;
        if (have) {
            const size_t e = (size_t)v * g.nb + k;
            P = __ldg(g.rays + e);
            if constexpr (NCH == 2) {
                sv = ldg2(sn + e);
                if constexpr (SG == 2) sv1 = count > 1 ? ldg2(sn1 + e) : make_float2(0.f, 0.f);
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
            const long long q = ray_pos(P, bi) - a0q;
            const float wr = ray_w(P) * sscale;
            const int at = __popc(mask & ((1u << lane) - 1u));
            st_ray[w][at] = make_int4((int)(unsigned)(unsigned long long)q, (int)(q >> 32), P.z, __float_as_int(wr * sv.x));
            if constexpr (SG == 1)
                st_wp[w][at] = wr * sv.y;
            else
                st_w2[w][at] = make_float4(wr * sv.x, wr * sv.y, wr * sv1.x, wr * sv1.y);
        }
        const int nr = (n + kSwUnroll - 1) / kSwUnroll * kSwUnroll;
        if (lane >= n && lane < nr) {  // null rays pad the stage to a multiple of kSwUnroll
            st_ray[w][lane] = make_int4(0, -1000 << 2, 0, 0);
            if constexpr (SG == 1)
                st_wp[w][lane] = 0.f;
            else
                st_w2[w][lane] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
        // advance the cursor and fetch the next chunk while this one is processed
        k0 += 32;
        if (k0 > khi) {
            if (k2 <= k2hi) {
                k0 = k2;
                khi = k2hi;
                k2 = 1;
                k2hi = 0;
            } else {
                seek(v + G);
            }
        }
        fetch();
        __syncwarp();
        for (int r0 = 0; r0 < nr; r0 += kSwUnroll) {
            int hh[kSwUnroll];
            float ff[kSwUnroll], wc[kSwUnroll], wp[kSwUnroll];
            if constexpr (NCH == 2 && SG == 1) {  // w s_p of the block's rays: broadcast 16-byte loads
#pragma unroll
                for (int v4 = 0; v4 < kSwUnroll / 4; ++v4) {
                    const float4 p = *reinterpret_cast<const float4*>(&st_wp[w][r0 + 4 * v4]);
                    wp[4 * v4] = p.x;
                    wp[4 * v4 + 1] = p.y;
                    wp[4 * v4 + 2] = p.z;
                    wp[4 * v4 + 3] = p.w;
                }
            }
#pragma unroll
            for (int u = 0; u < kSwUnroll; ++u) {
                const int4 S = st_ray[w][r0 + u];
                const long long q = ((((long long)S.y) << 32) | (long long)(unsigned)S.x) + (long long)lane * S.z;
                hh[u] = pos_floor(q);
                ff[u] = frac_of(q);
                wc[u] = __int_as_float(S.w);
            }
            if constexpr (SG == 2) {
                // both slices' weights per ray; a row's four sums {c, p, c', p'} advance as two packed
                // float32 pairs (fma.rn.f32x2, each element rounded as fmaf)
#pragma unroll
                for (int u = 0; u < kSwUnroll; ++u) {
                    const float4 x = st_w2[w][r0 + u];
                    if ((unsigned)(hh[u] + 1) < (unsigned)(TILE + 1)) {
                        float4* a = &acc4[w][hh[u] + 1][lane];
                        const float4 x0 = a[0], x1 = a[32];
                        const f32x2 g0 = pack2(1.0f - ff[u], 1.0f - ff[u]), g1 = pack2(ff[u], ff[u]);
                        const f32x2 w01 = pack2(x.x, x.y), w23 = pack2(x.z, x.w);
                        const float2 y00 = unpack2(fma2(g0, w01, pack2(x0.x, x0.y)));
                        const float2 y01 = unpack2(fma2(g0, w23, pack2(x0.z, x0.w)));
                        const float2 y10 = unpack2(fma2(g1, w01, pack2(x1.x, x1.y)));
                        const float2 y11 = unpack2(fma2(g1, w23, pack2(x1.z, x1.w)));
                        a[0] = make_float4(y00.x, y00.y, y01.x, y01.y);
                        a[32] = make_float4(y10.x, y10.y, y11.x, y11.y);
                    }
                }
                continue;
            }
#pragma unroll
            for (int u = 0; u < kSwUnroll; ++u) {
                // rows h, h+1 with h in [-1, TILE - 1] are accumulator rows h+1, h+2 (lanes outside skip)
                if ((unsigned)(hh[u] + 1) < (unsigned)(TILE + 1)) {
                    Acc* a = &acc[w][hh[u] + 1][lane];
                    if constexpr (NCH == 2) {
                        float2 x0 = a[0], x1 = a[32];
                        x0.x = fmaf(1.0f - ff[u], wc[u], x0.x);
                        x0.y = fmaf(1.0f - ff[u], wp[u], x0.y);
                        x1.x = fmaf(ff[u], wc[u], x1.x);
                        x1.y = fmaf(ff[u], wp[u], x1.y);
                        a[0] = x0;
                        a[32] = x1;
                    } else {
                        a[0] = fmaf(1.0f - ff[u], wc[u], a[0]);
                        a[32] = fmaf(ff[u], wc[u], a[32]);
                    }
                }
            }
        }
        __syncwarp();  // the stage is rewritten by the next chunk
    }
    __syncthreads();
    if constexpr (CLUSTER) {
        namespace cg = cooperative_groups;
        cg::cluster_group cl = cg::this_cluster();
        cl.sync();  // every view group of the tile has finished its accumulators
        const int rank = (int)cl.block_rank(), nrank = (int)cl.num_blocks();
        for (int px = rank * (int)blockDim.x + (int)threadIdx.x; px < TILE * TILE; px += nrank * (int)blockDim.x) {
            const int rr = px / TILE, cc = px % TILE;
            const int i = ti + cc, j = tj + rr;
            if (i < nx && j < ny) {
                Acc sum{};
                for (int k = 0; k < nrank; ++k) {
                    Acc(*peer)[Sh::kRows][32] = cl.map_shared_rank(acc, k);
                    const Acc a = peer[cc / 32][rr + 1][cc % 32], b = peer[Sh::kBands + rr / 32][cc + 1][rr % 32];
                    if constexpr (NCH == 2) {
                        sum.x += a.x + b.x;
                        sum.y += a.y + b.y;
                    } else {
                        sum += a + b;
                    }
                }
                partial[d.img_off + (size_t)j * nx + i] = sum;
            }
        }
        cl.sync();  // the peers' shared memory stays valid until every rank has read it
    } else {
        for (int q = 0; q < count; ++q) {
            const int64_t off = c * stride + dsl[sl[q]].img_off;
            for (int px = threadIdx.x; px < TILE * TILE; px += blockDim.x) {
                const int rr = px / TILE, cc = px % TILE;
                const int i = ti + cc, j = tj + rr;
                if (i < nx && j < ny) {
                    Acc a, b;
                    if constexpr (SG == 2) {
                        const float4 a4 = acc4[cc / 32][rr + 1][cc % 32], b4 = acc4[Sh::kBands + rr / 32][cc + 1][rr % 32];
                        a = q == 0 ? make_float2(a4.x, a4.y) : make_float2(a4.z, a4.w);
                        b = q == 0 ? make_float2(b4.x, b4.y) : make_float2(b4.z, b4.w);
                    } else {
                        a = acc[cc / 32][rr + 1][cc % 32];
                        b = acc[Sh::kBands + rr / 32][cc + 1][rr % 32];
                    }
                    Acc sum{};
                    if constexpr (NCH == 2) {
                        sum.x += a.x + b.x;
                        sum.y += a.y + b.y;
                    } else {
                        sum += a + b;
                    }
                    partial[off + (size_t)j * nx + i] = sum;
                }
            }
        }
        if (tile_count == nullptr || C == 1) return;
        // reduced form: the CTA that completes the tile's count sees every other CTA's partial (each
        // fenced its stores before its increment)
        __shared__ int last;
        __threadfence();
        __syncthreads();
        if (threadIdx.x == 0) last = atomicAdd(tile_count + blockIdx.x / C, 1) == C - 1;
        __syncthreads();
        if (!last) return;
        __threadfence();
        const int iw = min(TILE, nx - ti), jh = min(TILE, ny - tj);
        // four pixels per thread at a time, their C partials loaded view group by view group, so that
        // several loads are in flight per thread; each pixel still adds its partials in order 0..C-1
        constexpr int U = 4;
        for (int q = 0; q < count; ++q) {
            Acc* img = partial + dsl[sl[q]].img_off;
            for (int px0 = threadIdx.x; px0 < TILE * TILE; px0 += U * blockDim.x) {
                size_t e[U];
                bool in[U];
                Acc sum[U];
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const int px = px0 + u * (int)blockDim.x;
                    const int rr = px / TILE, cc = px % TILE;
                    in[u] = px < TILE * TILE && cc < iw && rr < jh;
                    e[u] = in[u] ? (size_t)(tj + rr) * nx + ti + cc : 0;
                    sum[u] = Acc{};
                }
#pragma unroll 2
                for (int k = 0; k < C; ++k) {
#pragma unroll
                    for (int u = 0; u < U; ++u) {
                        if (!in[u]) continue;
                        const Acc a = __ldcg(img + k * stride + e[u]);
                        if constexpr (NCH == 2) {
                            sum[u].x += a.x;
                            sum[u].y += a.y;
                        } else {
                            sum[u] += a;
                        }
                    }
                }
#pragma unroll
                for (int u = 0; u < U; ++u)
                    if (in[u]) img[e[u]] = sum[u];
            }
        }
        __syncthreads();  // every partial of the tile has been read
        for (int t = threadIdx.x; t < count * (C - 1) * jh; t += blockDim.x) {
            const int rr = t % jh, k = 1 + (t / jh) % (C - 1), q = t / (jh * (C - 1));
            const Acc* row = partial + dsl[sl[q]].img_off + k * stride + (size_t)(tj + rr) * nx + ti;
            discard_l2_range(row, row + iw);
        }
        if (threadIdx.x == 0) tile_count[blockIdx.x / C] = 0;
    }
}

// (planar != nullptr: single slice, written as [nch][ny][nx] instead of interleaved into `out`)
// A block finishes the 256 pixels of its map block with fin_threads(MODE) threads, each taking pixels
// that many apart: four pixels per thread for the light epilogues (their stencil loads in flight
// together), one for r0's (measured faster with its larger register footprint).
__host__ __device__ constexpr int fin_threads(int mode) { return (mode == BP_R0 || mode == BP_R0_NOGRAD) ? 256 : 64; }
template <int MODE>
__global__ void __launch_bounds__(fin_threads(MODE)) k_bp_finalize(const SliceDesc* __restrict__ dsl, BlockMap pix,
                                                                   int C, const float2* __restrict__ partial,
                                                                   int64_t stride, float2* __restrict__ out,
                                                                   BpEpilogue ep, float* __restrict__ planar, int nch) {
    constexpr int kFinThreads = fin_threads(MODE);
    int local;
    const int s = slice_of(pix, blockIdx.x, local);
    const SliceDesc& d = dsl[s];
    const int64_t np = (int64_t)d.g.nx * d.g.ny;
    float dot_c = 0.f, dot_p = 0.f;
#pragma unroll
    for (int t = 0; t < 256 / kFinThreads; ++t) {
        const int64_t k = (int64_t)local * 256 + t * kFinThreads + threadIdx.x;
        if (k < np) {
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
    }
    if (MODE == BP_AP || MODE == BP_AP_NOGRAD) bp_block_dots(dot_c, dot_p, ep.partial);
}

int sweep_tiles(int nx, int ny, int tile) { return ((nx + tile - 1) / tile) * ((ny + tile - 1) / tile); }

int sweep_ctas_for_groups(int view_groups) { return view_groups; }
int sweep_groups_per_cta() { return 1; }

// the kernels' dynamic shared memory may exceed the default 48 KB (TILE 64); the attribute is per device
static std::mutex g_slots_mu;
static std::vector<int> g_slots[2];  // resident CTA slots of k_bp_sweep per device, TILE 32 and 64

template <class S2, int NCH, int TILE, bool CLUSTER, int SG>
static cudaError_t sweep_attr1() {
    auto* k = k_bp_sweep<S2, NCH, TILE, CLUSTER, SG>;
    cudaError_t e =
        cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sweep_acc_bytes<TILE, NCH, SG>());
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
    if (e == cudaSuccess && CLUSTER) e = cudaFuncSetAttribute(k, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    return e;
}

template <class S2, int NCH, int TILE>
static cudaError_t sweep_attr() {
    cudaError_t e = sweep_attr1<S2, NCH, TILE, false, 1>();
    if (e == cudaSuccess) e = sweep_attr1<S2, NCH, TILE, true, 1>();
    if constexpr (NCH == 2)
        if (e == cudaSuccess) e = sweep_attr1<S2, NCH, TILE, false, 2>();
    return e;
}

cudaError_t sweep_init_attributes() {
    cudaError_t e = cudaSuccess;
    for (cudaError_t r : {sweep_attr<float2, 2, 32>(), sweep_attr<__half2, 2, 32>(), sweep_attr<__nv_bfloat162, 2, 32>(),
                          sweep_attr<float, 1, 32>(), sweep_attr<float2, 2, 64>(), sweep_attr<__half2, 2, 64>(),
                          sweep_attr<__nv_bfloat162, 2, 64>(), sweep_attr<float, 1, 64>()})
        if (e == cudaSuccess) e = r;
    return e;
}

// CTA groups (view groups) per tile: the smallest C (up to 8) whose grid of tiles * C blocks fills the
// resident slots best.
int sweep_groups(int tiles, int tile) {
    int dev = 0;
    cudaGetDevice(&dev);
    const int which = tile == 64 ? 1 : 0;
    std::unique_lock<std::mutex> lk(g_slots_mu);
    if ((int)g_slots[which].size() <= dev) g_slots[which].resize(dev + 1, 0);
    if (!g_slots[which][dev]) {
        int sms = 0, occ = 0;
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        sweep_init_attributes();
        if (which)
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_bp_sweep<float2, 2, 64>, SweepShape<64>::kThreads,
                                                          sweep_acc_bytes<64, 2>());
        else
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_bp_sweep<float2, 2, 32>, SweepShape<32>::kThreads,
                                                          sweep_acc_bytes<32, 2>());
        g_slots[which][dev] = sms * (occ > 0 ? occ : 1);
    }
    const int slots = g_slots[which][dev];
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

template <class S2, int NCH, int TILE>
static void sweep_t(const SliceDesc* dsl, const BlockMap& smap, int nsweep, int C, bool cluster, int sg,
                    const int4* groups, const S2* sino, typename std::conditional<NCH == 2, float2, float>::type* partial,
                    int64_t stride, const float* rw, const float* scale, int* tile_count, cudaStream_t st) {
    if constexpr (NCH == 2) {
        if (sg == 2) {
            k_bp_sweep<S2, NCH, TILE, false, 2><<<nsweep, SweepShape<TILE>::kThreads, sweep_acc_bytes<TILE, NCH, 2>(), st>>>(
                dsl, smap, C, groups, sino, partial, stride, rw, scale, tile_count);
            return;
        }
    }
    if (!cluster || C == 1) {
        k_bp_sweep<S2, NCH, TILE><<<nsweep, SweepShape<TILE>::kThreads, sweep_acc_bytes<TILE, NCH>(), st>>>(
            dsl, smap, C, nullptr, sino, partial, stride, rw, scale, tile_count);
        return;
    }
    // the C CTAs of a tile are consecutive blocks and every slice's block range is a multiple of C,
    // so a cluster of C blocks is exactly one tile's view groups
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)nsweep);
    cfg.blockDim = dim3(SweepShape<TILE>::kThreads);
    cfg.dynamicSmemBytes = sweep_acc_bytes<TILE, NCH>();
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    const int4* no_groups = nullptr;
    int* no_count = nullptr;
    cudaLaunchKernelEx(&cfg, k_bp_sweep<S2, NCH, TILE, true>, dsl, smap, C, no_groups, sino, partial, stride, rw,
                       scale, no_count);
}

void launch_bp_sweep(const SliceDesc* dsl, const BlockMap& smap, int nsweep, int C, int tile, bool cluster, int sg,
                     const int4* groups, const void* sino, float2* partial, int64_t stride, int prec, int* tile_count,
                     cudaStream_t st) {
    const bool k = cluster;
    int* tc = cluster ? nullptr : tile_count;
    if (tile == 64) {
        if (prec == PREC_F16)
            sweep_t<__half2, 2, 64>(dsl, smap, nsweep, C, k, sg, groups, (const __half2*)sino, partial, stride, nullptr,
                                    nullptr, tc, st);
        else if (prec == PREC_BF16)
            sweep_t<__nv_bfloat162, 2, 64>(dsl, smap, nsweep, C, k, sg, groups, (const __nv_bfloat162*)sino, partial,
                                           stride, nullptr, nullptr, tc, st);
        else
            sweep_t<float2, 2, 64>(dsl, smap, nsweep, C, k, sg, groups, (const float2*)sino, partial, stride, nullptr,
                                   nullptr, tc, st);
    } else {
        if (prec == PREC_F16)
            sweep_t<__half2, 2, 32>(dsl, smap, nsweep, C, k, sg, groups, (const __half2*)sino, partial, stride, nullptr,
                                    nullptr, tc, st);
        else if (prec == PREC_BF16)
            sweep_t<__nv_bfloat162, 2, 32>(dsl, smap, nsweep, C, k, sg, groups, (const __nv_bfloat162*)sino, partial,
                                           stride, nullptr, nullptr, tc, st);
        else
            sweep_t<float2, 2, 32>(dsl, smap, nsweep, C, k, sg, groups, (const float2*)sino, partial, stride, nullptr,
                                   nullptr, tc, st);
    }
}

void launch_bp_sweep1(const SliceDesc* dsl, const BlockMap& smap, int nsweep, int C, int tile, bool cluster,
                      const float* sino, const float* rw, const float* scale, float* partial, int64_t stride,
                      int* tile_count, cudaStream_t st) {
    int* tc = cluster ? nullptr : tile_count;
    if (tile == 64)
        sweep_t<float, 1, 64>(dsl, smap, nsweep, C, cluster, 1, nullptr, sino, partial, stride, rw, scale, tc, st);
    else
        sweep_t<float, 1, 32>(dsl, smap, nsweep, C, cluster, 1, nullptr, sino, partial, stride, rw, scale, tc, st);
}

template <int MODE>
static void finalize_t(const SliceDesc* dsl, const BlockMap& pix, int npix, int C, const float2* partial,
                       int64_t stride, float2* out, const BpEpilogue& ep, cudaStream_t st) {
    k_bp_finalize<MODE><<<npix, fin_threads(MODE), 0, st>>>(dsl, pix, C, partial, stride, out, ep, nullptr, 0);
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

void backproject_single(const SliceDesc& sd, const SliceDesc* d_dev, const int* maps, int C, int tile, const float* sino,
                        int nch, float2* packed, float2* partial, float* out, cudaStream_t st) {
    const int64_t nr = (int64_t)sd.g.nv * sd.g.nb, np = (int64_t)sd.g.nx * sd.g.ny;
    launch_pack_planar(sino, nch, nr, packed, st);
    const BlockMap smap{maps, 1}, pmap{maps + 2, 1};
    launch_bp_sweep(d_dev, smap, sweep_tiles(sd.g.nx, sd.g.ny, tile) * C, C, tile, false, 1, nullptr, packed, partial,
                    np, PREC_F32, nullptr, st);
    k_bp_finalize<BP_PLAIN><<<(unsigned)((np + 255) / 256), fin_threads(BP_PLAIN), 0, st>>>(d_dev, pmap, C, partial, np, nullptr,
                                                                         BpEpilogue{}, out, nch);
}

}  // namespace dect
