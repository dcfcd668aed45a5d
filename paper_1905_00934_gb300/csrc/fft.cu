// Preconditioner of the Eq. 12 conjugate-gradient solve (Sec. 3.3: the system
// is shift-invariant once the statistical weights move into the decomposition
// step, so it is preconditioned by a high-pass filter applied by FFT).
//
// M^-1 r = crop(IDFT2(H * DFT2(zero-pad(r)))) on a [py][px] grid (powers of two
// >= 2N). H is real and even, so one complex transform carries both bases:
// the Compton image in the real part and the PE image in the imaginary part.
// Three kernels: forward row FFTs of the ny non-zero rows; per column group a
// forward column FFT, the multiplication by H and the inverse column FFT (rows
// >= ny are known zeros on input and are not needed on output); inverse row
// FFTs of the ny rows, cropped to nx, fused with the partial sums of <r, s>.
// The FFTs are radix 2 with a float32 twiddle table computed once in float64
// on the host. An axis whose padded length is 64..2048 splits, by its zero
// upper half, into two half-length FFTs held in the registers of a warp pair
// (forward by decimation in frequency, inverse by decimation in time, so no
// bit-reversal pass); other lengths, and the response's forward transform, use
// decimation in time staged through shared memory.
#include <cuda_runtime.h>
#include <math.h>

#include <mutex>
#include <vector>

#include "dect_internal.cuh"

namespace dect {

static std::mutex g_tw_mu;
static std::vector<float2*> g_tw;  // per device

const float2* fft_twiddles() {
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lk(g_tw_mu);
    if ((int)g_tw.size() <= dev) g_tw.resize(dev + 1, nullptr);
    if (!g_tw[dev]) {
        std::vector<float2> h(kFftMax / 2);
        for (int t = 0; t < kFftMax / 2; ++t) {
            const double th = 2.0 * M_PI * (double)t / (double)kFftMax;
            h[t] = make_float2((float)cos(th), (float)(-sin(th)));
        }
        float2* d = nullptr;
        if (cudaMalloc(&d, sizeof(float2) * h.size()) != cudaSuccess) return nullptr;
        if (cudaMemcpy(d, h.data(), sizeof(float2) * h.size(), cudaMemcpyHostToDevice) != cudaSuccess) {
            cudaFree(d);
            return nullptr;
        }
        g_tw[dev] = d;
    }
    return g_tw[dev];
}

__device__ __forceinline__ int bitrev(int t, int logn) { return (int)(__brev((unsigned)t) >> (32 - logn)); }

// Shared staging of the register-path FFTs: one float2 of padding after every 32, and columns S(py)
// apart, so the bit-reversed scatters and gathers spread over the banks (8-byte accesses: 2 to 4
// wavefronts per warp instead of up to 32). The layout moves data only; the arithmetic is unchanged.
__host__ __device__ __forceinline__ int spad(int p) { return p + (p >> 5); }
__host__ __device__ constexpr int col_stride(int py) { return py + py / 32 + 2; }
constexpr int kColsSmem = 8 * col_stride(1024);  // float2 entries: 8 padded columns of up to 1024 rows
static_assert(kColsSmem >= 8192, "the shared-memory path stages C(py) * py <= 8192 entries");

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}

// In-place FFT of length 2^logn on a bit-reversed shared buffer; `lane`/`nlanes` split the butterflies.
// Every thread of the block must call it (it synchronises the block after each stage).
__device__ void fft_stages(float2* buf, int logn, bool inverse, const float2* __restrict__ tw, int lane, int nlanes) {
    const int n = 1 << logn;
    for (int s = 0; s < logn; ++s) {
        const int half = 1 << s;
        const int stride = kFftMax >> (s + 1);
        for (int b = lane; b < n / 2; b += nlanes) {
            const int pos = b & (half - 1);
            const int i0 = ((b >> s) << (s + 1)) + pos;
            const int i1 = i0 + half;
            float2 w = __ldg(tw + pos * stride);
            if (inverse) w.y = -w.y;
            const float2 x0 = buf[i0];
            const float2 t = cmul(w, buf[i1]);
            buf[i0] = make_float2(x0.x + t.x, x0.y + t.y);
            buf[i1] = make_float2(x0.x - t.x, x0.y - t.y);
        }
        __syncthreads();
    }
}

// In-place bit-reversal permutation of a shared buffer (natural <-> bit-reversed order).
__device__ void bitrev_permute(float2* buf, int logn, int lane, int nlanes) {
    const int n = 1 << logn;
    for (int t = lane; t < n; t += nlanes) {
        const int r = bitrev(t, logn);
        if (t < r) {
            const float2 a = buf[t];
            buf[t] = buf[r];
            buf[r] = a;
        }
    }
    __syncthreads();
}

__host__ __device__ int precond_cols_per_block(int py) { return py >= 4096 ? 2 : (py >= 2048 ? 4 : 8); }

// ---- column frequencies of the row pass's output -------------------------------------------------
// The split row pass (px in 64..2048) stores a row's spectrum half by half, each half in bit-reversed
// order: storage column k holds frequency 2 * bitrev(k mod px/2) + (k >= px/2). Otherwise storage column
// k holds frequency k.
__device__ __forceinline__ int col_freq(int k, int px, int lpx) {
    if (!precond_split(px)) return k;
    const int hh = px >> 1;
    return 2 * bitrev(k & (hh - 1), lpx - 1) + (k >= hh ? 1 : 0);
}

// W_P^i = exp(-2 pi i i / P) (conjugated for the inverse), P = 2^lp <= kFftMax, i < P / 2
__device__ __forceinline__ float2 tw_pow(const float2* __restrict__ tw, int i, int lp, bool inverse) {
    float2 w = __ldg(tw + (i << (kFftMaxLog2 - lp)));
    if (inverse) w.y = -w.y;
    return w;
}

// barrier of the two warps (64 threads) of pair q of a 256-thread block (named barriers 1..4)
__device__ __forceinline__ void pair_sync(int q) { asm volatile("bar.sync %0, 64;" ::"r"(q + 1) : "memory"); }

static int ilog2_int(int v) {
    int l = 0;
    while ((1 << (l + 1)) <= v) ++l;
    return l;
}


// The same radix-2 DIT FFT (same butterflies, twiddles and operation order, so the same results) held
// in registers by one warp, for lengths 2^LOG with 5 <= LOG <= 10: lane t holds elements 32 m + t of the
// bit-reversed sequence in v[m]. Stages with half < 32 pair lanes t and t ^ half (shuffles); stages with
// half >= 32 pair slots m and m + half/32 of the same lane. No shared memory, no barriers.
template <int LOG>
__device__ __forceinline__ void fft_warp_regs(float2 (&v)[1 << (LOG - 5)], int lane, bool inverse,
                                              const float2* __restrict__ tw) {
    constexpr int M = 1 << (LOG - 5);
#pragma unroll
    for (int s = 0; s < 5; ++s) {
        const int half = 1 << s;
        float2 w = __ldg(tw + (lane & (half - 1)) * (kFftMax >> (s + 1)));
        if (inverse) w.y = -w.y;
        const bool upper = (lane & half) != 0;
#pragma unroll
        for (int m = 0; m < M; ++m) {
            const float2 o = make_float2(__shfl_xor_sync(0xffffffffu, v[m].x, half),
                                         __shfl_xor_sync(0xffffffffu, v[m].y, half));
            const float2 x0 = upper ? o : v[m];
            const float2 t = cmul(w, upper ? v[m] : o);
            v[m] = upper ? make_float2(x0.x - t.x, x0.y - t.y) : make_float2(x0.x + t.x, x0.y + t.y);
        }
    }
#pragma unroll
    for (int s = 5; s < LOG; ++s) {
        const int hs = 1 << (s - 5);
#pragma unroll
        for (int m = 0; m < M; ++m) {
            if (m & hs) continue;
            float2 w = __ldg(tw + (((m & (hs - 1)) << 5) + lane) * (kFftMax >> (s + 1)));
            if (inverse) w.y = -w.y;
            const float2 x0 = v[m];
            const float2 t = cmul(w, v[m + hs]);
            v[m] = make_float2(x0.x + t.x, x0.y + t.y);
            v[m + hs] = make_float2(x0.x - t.x, x0.y - t.y);
        }
    }
}

// Forward FFT of the same lengths by decimation in frequency, in registers: lane t holds element 32 m + t
// of the natural-order sequence in v[m] on entry and element 32 m + t of the bit-reversed spectrum on
// return (the order the inverse fft_warp_regs takes). Butterflies x0 + x1 and W (x0 - x1), the longest
// stride first: the stages with half >= 32 within a lane, then the five shuffle stages.
template <int LOG>
__device__ __forceinline__ void fft_warp_regs_dif(float2 (&v)[1 << (LOG - 5)], int lane, const float2* __restrict__ tw) {
    constexpr int M = 1 << (LOG - 5);
#pragma unroll
    for (int s = LOG - 1; s >= 5; --s) {
        const int hs = 1 << (s - 5);
#pragma unroll
        for (int m = 0; m < M; ++m) {
            if (m & hs) continue;
            const float2 w = __ldg(tw + (((m & (hs - 1)) << 5) + lane) * (kFftMax >> (s + 1)));
            const float2 a = v[m], b = v[m + hs];
            v[m] = make_float2(a.x + b.x, a.y + b.y);
            v[m + hs] = cmul(w, make_float2(a.x - b.x, a.y - b.y));
        }
    }
#pragma unroll
    for (int s = 4; s >= 0; --s) {
        const int half = 1 << s;
        const float2 w = __ldg(tw + (lane & (half - 1)) * (kFftMax >> (s + 1)));
        const bool upper = (lane & half) != 0;
#pragma unroll
        for (int m = 0; m < M; ++m) {
            const float2 o = make_float2(__shfl_xor_sync(0xffffffffu, v[m].x, half),
                                         __shfl_xor_sync(0xffffffffu, v[m].y, half));
            // the lower lane keeps x0 + x1, the upper lane W (x0 - x1), x0 being the lower lane's value
            v[m] = upper ? cmul(w, make_float2(o.x - v[m].x, o.y - v[m].y)) : make_float2(v[m].x + o.x, v[m].y + o.y);
        }
    }
}

// Column group of k_fft_cols on the register path: 8 columns, warp c owns column c (blockDim 256).
// buf holds the group's columns in bit-reversed order on entry; on return, rows in natural order.
// Columns in the padded layout: column c at buf + c * col_stride(py), row j at spad(j).
template <int LOG>
__device__ void cols_regs(float2* buf, const float* __restrict__ hs, int px, int lpx, int k0,
                          const float2* __restrict__ tw) {
    constexpr int M = 1 << (LOG - 5), py = 1 << LOG, C = 8, S = col_stride(py);
    const int c = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float2* col = buf + c * S;
    float2 v[M];
#pragma unroll
    for (int m = 0; m < M; ++m) v[m] = col[spad((m << 5) + lane)];
    fft_warp_regs<LOG>(v, lane, false, tw);
    if (hs) {
#pragma unroll
        for (int m = 0; m < M; ++m) col[spad((m << 5) + lane)] = v[m];
        __syncthreads();
        for (int e = threadIdx.x; e < C * py; e += blockDim.x) {
            const int cc = e % C, j = e / C;
            const int k = k0 + cc;
            const float h = k < px ? __ldg(hs + (size_t)j * px + col_freq(k, px, lpx)) : 0.f;
            float2& x = buf[cc * S + spad(j)];
            x.x *= h;
            x.y *= h;
        }
        __syncthreads();
#pragma unroll
        for (int m = 0; m < M; ++m) v[m] = col[spad(bitrev((m << 5) + lane, LOG))];
        fft_warp_regs<LOG>(v, lane, true, tw);
    }
    // every lane has passed the shuffles above, so all reads of this column are done
#pragma unroll
    for (int m = 0; m < M; ++m) col[spad((m << 5) + lane)] = v[m];
}



// ---- fallback paths (padded length 32 or >= 4096): shared-memory stages, one row or C(py) columns -----

__device__ void row_fwd_staged(const SliceDesc& d, int j, const float2* __restrict__ r, float2* __restrict__ Z,
                               const float2* __restrict__ tw, float2* buf) {
    const int px = d.px, lp = d.lpx, nx = d.g.nx;
    const float2* row = r + d.img_off + (size_t)j * nx;
    for (int t = threadIdx.x; t < px; t += blockDim.x)
        buf[bitrev(t, lp)] = t < nx ? __ldg(row + t) : make_float2(0.f, 0.f);
    __syncthreads();
    fft_stages(buf, lp, false, tw, threadIdx.x, blockDim.x);
    float2* zr = Z + d.fft_off + (size_t)j * px;
    for (int t = threadIdx.x; t < px; t += blockDim.x) zr[t] = buf[t];
}

// per group of C(py) columns: forward column FFT (rows >= rows_in are zero), optional multiplication by
// H (at the column's frequency, col_freq), inverse column FFT; writes rows [0, rows_out). REGS: the
// register path for 64 <= py <= 1024 is compiled in (the apply path reaches this only for py = 32 or
// py >= 4096 and leaves it out, keeping its register count to the split path's).
template <bool REGS>
__device__ void cols_staged(const SliceDesc& d, int g, float2* __restrict__ Z, const float* __restrict__ H,
                            int rows_in_all, int rows_out_all, const float2* __restrict__ tw, float2* buf) {
    const int px = d.px, py = d.py, lp = d.lpy;
    const int C = precond_cols_per_block(py);
    const int k0 = g * C;
    const int rows_in = rows_in_all ? py : d.g.ny;
    const int rows_out = rows_out_all ? py : d.g.ny;
    float2* zs = Z + d.fft_off;
    // register path (32 <= py <= 1024): padded columns; otherwise columns py apart
    const bool regs = lp >= 5 && lp <= 10;
    const int S = regs ? col_stride(py) : py;
    // load: consecutive threads take consecutive columns of one row
    for (int e = threadIdx.x; e < C * py; e += blockDim.x) {
        const int c = e % C, j = e / C;
        const int k = k0 + c;
        float2 v = make_float2(0.f, 0.f);
        if (j < rows_in && k < px) v = zs[(size_t)j * px + k];
        const int jb = bitrev(j, lp);
        buf[c * S + (regs ? spad(jb) : jb)] = v;
    }
    __syncthreads();
    const float* hs = H ? H + d.h_off : nullptr;
    switch (lp) {  // one slice per block, so the branch is uniform
        case 5: cols_regs<5>(buf, hs, px, d.lpx, k0, tw); break;
        case 6: if constexpr (REGS) cols_regs<6>(buf, hs, px, d.lpx, k0, tw); break;
        case 7: if constexpr (REGS) cols_regs<7>(buf, hs, px, d.lpx, k0, tw); break;
        case 8: if constexpr (REGS) cols_regs<8>(buf, hs, px, d.lpx, k0, tw); break;
        case 9: if constexpr (REGS) cols_regs<9>(buf, hs, px, d.lpx, k0, tw); break;
        case 10: if constexpr (REGS) cols_regs<10>(buf, hs, px, d.lpx, k0, tw); break;
        default: {  // py < 32 or py >= 2048: shared-memory stages, C columns of blockDim/C threads each
            const int lanes = blockDim.x / C;
            const int c = threadIdx.x / lanes, lane = threadIdx.x % lanes;
            fft_stages(buf + c * py, lp, false, tw, lane, lanes);
            if (hs) {
                for (int e = threadIdx.x; e < C * py; e += blockDim.x) {
                    const int cc = e % C, j = e / C;
                    const int k = k0 + cc;
                    const float h = k < px ? __ldg(hs + (size_t)j * px + col_freq(k, px, d.lpx)) : 0.f;
                    float2& v = buf[cc * py + j];
                    v.x *= h;
                    v.y *= h;
                }
                __syncthreads();
                bitrev_permute(buf + c * py, lp, lane, lanes);
                fft_stages(buf + c * py, lp, true, tw, lane, lanes);
            }
        }
    }
    __syncthreads();
    for (int e = threadIdx.x; e < C * rows_out; e += blockDim.x) {
        const int cc = e % C, j = e / C;
        const int k = k0 + cc;
        if (k < px) zs[(size_t)j * px + k] = buf[cc * S + (regs ? spad(j) : j)];
    }
}

// inverse row FFT of row j, crop to nx, scale by 1/(px*py) into s_out; threads 0..31 return <r, s> of
// the row per channel (a lane's products in float32, the lanes in float64), the others zero
__device__ void row_inv_staged(const SliceDesc& d, int j, const float2* __restrict__ Z, const float2* __restrict__ r,
                               float2* __restrict__ s_out, const float2* __restrict__ tw, float2* buf, double& dc,
                               double& dp) {
    const int px = d.px, lp = d.lpx, nx = d.g.nx;
    const float2* zr = Z + d.fft_off + (size_t)j * px;
    for (int t = threadIdx.x; t < px; t += blockDim.x) buf[bitrev(t, lp)] = zr[t];
    __syncthreads();
    fft_stages(buf, lp, true, tw, threadIdx.x, blockDim.x);
    const float scale = 1.0f / ((float)px * (float)d.py);
    const size_t row = d.img_off + (size_t)j * nx;
    for (int t = threadIdx.x; t < nx; t += blockDim.x)
        s_out[row + t] = make_float2(buf[t].x * scale, buf[t].y * scale);
    dc = dp = 0.0;
    if (threadIdx.x < 32) {
        float fc = 0.f, fp = 0.f;
        for (int t = threadIdx.x; t < nx; t += 32) {
            const float2 v = make_float2(buf[t].x * scale, buf[t].y * scale);
            const float2 rv = __ldg(r + row + t);
            fc = fmaf(rv.x, v.x, fc);
            fp = fmaf(rv.y, v.y, fp);
        }
        dc = (double)fc;
        dp = (double)fp;
        for (int o = 16; o > 0; o >>= 1) {
            dc += __shfl_down_sync(0xffffffffu, dc, o);
            dp += __shfl_down_sync(0xffffffffu, dp, o);
        }
    }
}

// The response path's column pass (H = nullptr) and any caller of the staged column pass.
__global__ void __launch_bounds__(256) k_fft_cols(const SliceDesc* __restrict__ dsl, BlockMap map,
                                                  float2* __restrict__ Z, const float* __restrict__ H, int rows_in_all,
                                                  int rows_out_all, const float2* __restrict__ tw) {
    extern __shared__ float2 buf[];
    int g;
    const int s = slice_of(map, blockIdx.x, g);
    cols_staged<true>(dsl[s], g, Z, H, rows_in_all, rows_out_all, tw, buf);
}

// ---- the preconditioner's apply path: split-half register FFTs ----------------------------------------
// Along an axis of padded length P (64..2048) only the first P/2 entries are non-zero (the grid pads
// each image axis at least twice), so the length-P spectrum splits exactly into two length-P/2 ones:
// X[2f + h] = DFT_{P/2}(x[i] W_P^{h i})[f], h = 0, 1. A pair of warps holds one row or column, warp h
// computing half h in registers (fft_warp_regs_dif: natural order in, bit-reversed out). The inverse
// takes each half back with fft_warp_regs (bit-reversed in, natural out) and recombines:
// x[n] = z_0[n] + W_P^{-n} z_1[n] for the n < P/2 that are kept. A 256-thread block holds 4 pairs.
// Slices with another padded length use the staged paths above in the same launch (one row, or C(py)
// columns, per block); the choice depends on the slice alone.

template <int L>
__device__ __forceinline__ void split_row_fwd(const float2* __restrict__ row, int nx, float2* __restrict__ zr, int h,
                                              const float2* __restrict__ tw) {
    constexpr int M = 1 << (L - 5), HH = 1 << L;
    const int lane = threadIdx.x & 31;
    float2 v[M];
#pragma unroll
    for (int m = 0; m < M; ++m) {
        const int i = (m << 5) + lane;
        const float2 x = i < nx ? __ldg(row + i) : make_float2(0.f, 0.f);
        v[m] = h ? cmul(tw_pow(tw, i, L + 1, false), x) : x;
    }
    fft_warp_regs_dif<L>(v, lane, tw);
#pragma unroll
    for (int m = 0; m < M; ++m) zr[h * HH + (m << 5) + lane] = v[m];
}

// forward row FFTs of the image rows (Compton + i PE), zero-padded to px: split rows 4 per block,
// others one per block
template <int LMAX>
__global__ void __launch_bounds__(256) k_prec_rows_fwd(const SliceDesc* __restrict__ dsl, BlockMap map,
                                                       const float2* __restrict__ r, float2* __restrict__ Z,
                                                       const float2* __restrict__ tw) {
    extern __shared__ float2 buf[];
    int blk;
    const int s = slice_of(map, blockIdx.x, blk);
    const SliceDesc& d = dsl[s];
    if (!precond_split(d.px)) {
        row_fwd_staged(d, blk, r, Z, tw, buf);
        return;
    }
    const int q = threadIdx.x >> 6, h = (threadIdx.x >> 5) & 1;
    const int j = blk * 4 + q;
    if (j >= d.g.ny) return;  // warp-uniform; this path has no barriers
    const float2* row = r + d.img_off + (size_t)j * d.g.nx;
    float2* zr = Z + d.fft_off + (size_t)j * d.px;
    switch (d.lpx - 1) {
        case 5: split_row_fwd<5>(row, d.g.nx, zr, h, tw); break;
        case 6: split_row_fwd<(LMAX < 6 ? LMAX : 6)>(row, d.g.nx, zr, h, tw); break;
        case 7: split_row_fwd<(LMAX < 7 ? LMAX : 7)>(row, d.g.nx, zr, h, tw); break;
        case 8: split_row_fwd<(LMAX < 8 ? LMAX : 8)>(row, d.g.nx, zr, h, tw); break;
        case 9: split_row_fwd<(LMAX < 9 ? LMAX : 9)>(row, d.g.nx, zr, h, tw); break;
        default: split_row_fwd<LMAX>(row, d.g.nx, zr, h, tw); break;
    }
}

// Column pair q of the block: staged column c = q in buf (padded, natural row order, rows < ny), Hp the
// slice's permuted response (Hp[k][h P/2 + t] = H at row frequency 2 bitrev(t) + h, column frequency
// col_freq(k)); the recombined column is written back to its staging column.
template <int L>
__device__ __forceinline__ void split_col(float2* col, const float* __restrict__ hp, int ny, int h, int q,
                                          const float2* __restrict__ tw) {
    constexpr int M = 1 << (L - 5), HH = 1 << L;
    const int lane = threadIdx.x & 31;
    float2 v[M];
#pragma unroll
    for (int m = 0; m < M; ++m) {
        const int j = (m << 5) + lane;
        const float2 x = j < ny ? col[spad(j)] : make_float2(0.f, 0.f);
        v[m] = h ? cmul(tw_pow(tw, j, L + 1, false), x) : x;
    }
    pair_sync(q);  // both warps hold the column: its staging may be overwritten below
    fft_warp_regs_dif<L>(v, lane, tw);
#pragma unroll
    for (int m = 0; m < M; ++m) {
        const float hv = __ldg(hp + h * HH + (m << 5) + lane);
        v[m].x *= hv;
        v[m].y *= hv;
    }
    fft_warp_regs<L>(v, lane, true, tw);
    if (h) {
#pragma unroll
        for (int m = 0; m < M; ++m) {
            const int n = (m << 5) + lane;
            if (n < ny) col[spad(n)] = cmul(tw_pow(tw, n, L + 1, true), v[m]);
        }
    }
    pair_sync(q);
    if (!h) {
#pragma unroll
        for (int m = 0; m < M; ++m) {
            const int n = (m << 5) + lane;
            if (n < ny) {
                const float2 t = col[spad(n)];
                col[spad(n)] = make_float2(v[m].x + t.x, v[m].y + t.y);
            }
        }
    }
}

// the column pass of the apply: split columns 4 per block (staged through padded shared memory so the
// loads and stores take 4 neighbouring columns of a row), others C(py) per block (cols_staged)
template <int LMAX>
__global__ void __launch_bounds__(256) k_prec_cols(const SliceDesc* __restrict__ dsl, BlockMap map,
                                                   float2* __restrict__ Z, const float* __restrict__ H,
                                                   const float* __restrict__ Hp, const float2* __restrict__ tw) {
    extern __shared__ float2 buf[];
    int g;
    const int s = slice_of(map, blockIdx.x, g);
    const SliceDesc& d = dsl[s];
    if (!precond_split(d.py)) {
        cols_staged<false>(d, g, Z, H, 0, 0, tw, buf);
        return;
    }
    const int px = d.px, ny = d.g.ny, k0 = g * 4;
    const int S = spad(d.py >> 1) + 2;  // padded staging column
    float2* zs = Z + d.fft_off;
    for (int e = threadIdx.x; e < 4 * ny; e += blockDim.x) {
        const int c = e & 3, j = e >> 2, k = k0 + c;
        buf[c * S + spad(j)] = k < px ? zs[(size_t)j * px + k] : make_float2(0.f, 0.f);
    }
    __syncthreads();
    const int q = threadIdx.x >> 6, h = (threadIdx.x >> 5) & 1;
    const int k = k0 + q;
    if (k < px) {  // pair-uniform
        float2* col = buf + q * S;
        const float* hp = Hp + d.h_off + (size_t)k * d.py;
        switch (d.lpy - 1) {
            case 5: split_col<5>(col, hp, ny, h, q, tw); break;
            case 6: split_col<(LMAX < 6 ? LMAX : 6)>(col, hp, ny, h, q, tw); break;
            case 7: split_col<(LMAX < 7 ? LMAX : 7)>(col, hp, ny, h, q, tw); break;
            case 8: split_col<(LMAX < 8 ? LMAX : 8)>(col, hp, ny, h, q, tw); break;
            case 9: split_col<(LMAX < 9 ? LMAX : 9)>(col, hp, ny, h, q, tw); break;
            default: split_col<LMAX>(col, hp, ny, h, q, tw); break;
        }
    }
    __syncthreads();
    for (int e = threadIdx.x; e < 4 * ny; e += blockDim.x) {
        const int c = e & 3, j = e >> 2, k = k0 + c;
        if (k < px) zs[(size_t)j * px + k] = buf[c * S + spad(j)];
    }
}

// Row pair q: inverse of the split row spectrum, recombined, cropped to nx and scaled into s_out; the
// pair's first warp returns <r, s> of the row per channel (lane products in float32, lanes in float64).
template <int L>
__device__ __forceinline__ void split_row_inv(const float2* __restrict__ zr, const float2* __restrict__ rr,
                                              float2* __restrict__ so, int nx, float scale, int h, int q, float2* ex,
                                              const float2* __restrict__ tw, double& dc, double& dp) {
    constexpr int M = 1 << (L - 5), HH = 1 << L;
    const int lane = threadIdx.x & 31;
    float2 v[M];
#pragma unroll
    for (int m = 0; m < M; ++m) v[m] = zr[h * HH + (m << 5) + lane];
    fft_warp_regs<L>(v, lane, true, tw);
    if (h) {
#pragma unroll
        for (int m = 0; m < M; ++m) {
            const int n = (m << 5) + lane;
            if (n < nx) ex[n] = cmul(tw_pow(tw, n, L + 1, true), v[m]);
        }
    }
    pair_sync(q);
    dc = dp = 0.0;
    if (!h) {
        float fc = 0.f, fp = 0.f;
#pragma unroll
        for (int m = 0; m < M; ++m) {
            const int n = (m << 5) + lane;
            if (n < nx) {
                const float2 t = ex[n];
                const float2 x = make_float2((v[m].x + t.x) * scale, (v[m].y + t.y) * scale);
                so[n] = x;
                const float2 rv = __ldg(rr + n);
                fc = fmaf(rv.x, x.x, fc);
                fp = fmaf(rv.y, x.y, fp);
            }
        }
        dc = (double)fc;
        dp = (double)fp;
        for (int o = 16; o > 0; o >>= 1) {
            dc += __shfl_down_sync(0xffffffffu, dc, o);
            dp += __shfl_down_sync(0xffffffffu, dp, o);
        }
    }
}

// inverse row FFTs, crop to nx, scale by 1/(px*py): s = {Re, Im}; one partial <r, s> per block and
// channel (split rows: the block's 4 rows added in order)
template <int LMAX>
__global__ void __launch_bounds__(256) k_prec_rows_inv(const SliceDesc* __restrict__ dsl, BlockMap map,
                                                       const float2* __restrict__ Z, const float2* __restrict__ r,
                                                       float2* __restrict__ s_out, double* __restrict__ partial,
                                                       const float2* __restrict__ tw) {
    extern __shared__ float2 buf[];
    __shared__ double red[4][2];
    int blk;
    const int s = slice_of(map, blockIdx.x, blk);
    const SliceDesc& d = dsl[s];
    double dc = 0.0, dp = 0.0;
    if (!precond_split(d.px)) {
        row_inv_staged(d, blk, Z, r, s_out, tw, buf, dc, dp);
        if (threadIdx.x == 0) {
            partial[2 * (size_t)blockIdx.x] = dc;
            partial[2 * (size_t)blockIdx.x + 1] = dp;
        }
        return;
    }
    const int q = threadIdx.x >> 6, h = (threadIdx.x >> 5) & 1;
    const int j = blk * 4 + q;
    if (j < d.g.ny) {  // pair-uniform
        const float scale = 1.0f / ((float)d.px * (float)d.py);
        const float2* zr = Z + d.fft_off + (size_t)j * d.px;
        const size_t row = d.img_off + (size_t)j * d.g.nx;
        float2* ex = buf + q * (d.px >> 1);
        switch (d.lpx - 1) {
            case 5: split_row_inv<5>(zr, r + row, s_out + row, d.g.nx, scale, h, q, ex, tw, dc, dp); break;
            case 6: split_row_inv<(LMAX < 6 ? LMAX : 6)>(zr, r + row, s_out + row, d.g.nx, scale, h, q, ex, tw, dc, dp); break;
            case 7: split_row_inv<(LMAX < 7 ? LMAX : 7)>(zr, r + row, s_out + row, d.g.nx, scale, h, q, ex, tw, dc, dp); break;
            case 8: split_row_inv<(LMAX < 8 ? LMAX : 8)>(zr, r + row, s_out + row, d.g.nx, scale, h, q, ex, tw, dc, dp); break;
            case 9: split_row_inv<(LMAX < 9 ? LMAX : 9)>(zr, r + row, s_out + row, d.g.nx, scale, h, q, ex, tw, dc, dp); break;
            default: split_row_inv<LMAX>(zr, r + row, s_out + row, d.g.nx, scale, h, q, ex, tw, dc, dp); break;
        }
    }
    if ((threadIdx.x & 63) == 0) {
        red[q][0] = dc;
        red[q][1] = dp;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        partial[2 * (size_t)blockIdx.x] = ((red[0][0] + red[1][0]) + red[2][0]) + red[3][0];
        partial[2 * (size_t)blockIdx.x + 1] = ((red[0][1] + red[1][1]) + red[2][1]) + red[3][1];
    }
}

// Hp of a slice with a split column pass: Hp[k][h py/2 + t] = H[2 bitrev(t) + h][col_freq(k)]
__global__ void k_permute_response(SliceDesc d, const float* __restrict__ H, float* __restrict__ Hp) {
    const int64_t n = (int64_t)d.px * d.py;
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    const int k = (int)(e / d.py), qy = (int)(e % d.py);
    const int hh = d.py >> 1;
    const int ky = 2 * bitrev(qy & (hh - 1), d.lpy - 1) + (qy >= hh ? 1 : 0);
    Hp[e] = H[(size_t)ky * d.px + col_freq(k, d.px, d.lpx)];
}

void launch_permute_response(const SliceDesc& d, const float* H, float* Hp, cudaStream_t st) {
    if (!precond_split(d.py)) return;
    const int64_t n = (int64_t)d.px * d.py;
    k_permute_response<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(d, H + d.h_off, Hp + d.h_off);
}

template <int LMAX>
static void precond_t(const SliceDesc* dsl, const BlockMap& rows_map, int nrows_blk, const BlockMap& cols_map,
                      int ncols_blk, const float* H, const float* Hp, const float2* r, float2* s, float2* Z,
                      double* partial_rs, const float2* tw, size_t smem_fwd, size_t smem_cols, size_t smem_inv,
                      cudaStream_t st) {
    k_prec_rows_fwd<LMAX><<<nrows_blk, 256, smem_fwd, st>>>(dsl, rows_map, r, Z, tw);
    k_prec_cols<LMAX><<<ncols_blk, 256, smem_cols, st>>>(dsl, cols_map, Z, H, Hp, tw);
    k_prec_rows_inv<LMAX><<<nrows_blk, 256, smem_inv, st>>>(dsl, rows_map, Z, r, s, partial_rs, tw);
}

void launch_precond(const SliceDesc* dsl, const BlockMap& rows_map, int nrows_blk, const BlockMap& cols_map,
                    int ncols_blk, const float* H, const float* Hp, const float2* r, float2* s, float2* Z,
                    double* partial_rs, const float2* tw, int max_px, int min_px, int max_py, int min_py,
                    cudaStream_t st) {
    // shared memory: the staged paths' row (px) or columns (kColsSmem) where some slice takes them; the
    // split paths' 4 padded staging columns and 4 half-rows of exchange
    const bool all_x = min_px >= 64 && max_px <= 2048, all_y = min_py >= 64 && max_py <= 2048;
    const size_t f2 = sizeof(float2);
    const size_t smem_fwd = all_x ? 0 : f2 * max_px;
    const size_t smem_inv = f2 * std::max(all_x ? 0 : max_px, 4 * (std::min(max_px, 2048) / 2));
    const size_t smem_cols = f2 * std::max(all_y ? 0 : kColsSmem, 4 * (spad(std::min(max_py, 2048) / 2) + 2));
    const int lmax = std::max(ilog2_int(std::min(std::max(max_px, max_py), 2048)) - 1, 5);
    if (lmax <= 8)
        precond_t<8>(dsl, rows_map, nrows_blk, cols_map, ncols_blk, H, Hp, r, s, Z, partial_rs, tw, smem_fwd, smem_cols,
                     smem_inv, st);
    else if (lmax == 9)
        precond_t<9>(dsl, rows_map, nrows_blk, cols_map, ncols_blk, H, Hp, r, s, Z, partial_rs, tw, smem_fwd, smem_cols,
                     smem_inv, st);
    else
        precond_t<10>(dsl, rows_map, nrows_blk, cols_map, ncols_blk, H, Hp, r, s, Z, partial_rs, tw, smem_fwd,
                      smem_cols, smem_inv, st);
}

// ---- response H from the point response of R^T R ---------------------------------------------

__global__ void k_embed_psf(SliceDesc d, const float2* __restrict__ psf, float2* __restrict__ Z) {
    const int64_t n = (int64_t)d.px * d.py;
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    const int k = (int)(e / d.px), l = (int)(e % d.px);
    // grid index (k, l) holds the response at pixel (jc + k, ic + l) modulo the padded size
    const int jc = d.g.ny / 2, ic = d.g.nx / 2;
    int j = k < d.py / 2 ? jc + k : jc + k - d.py;
    int i = l < d.px / 2 ? ic + l : ic + l - d.px;
    float v = 0.f;
    if (j >= 0 && j < d.g.ny && i >= 0 && i < d.g.nx) v = psf[(size_t)j * d.g.nx + i].x;
    Z[e] = make_float2(v, 0.f);
}

__global__ void __launch_bounds__(256) k_fft_rows_full(SliceDesc d, float2* __restrict__ Z,
                                                       const float2* __restrict__ tw) {
    extern __shared__ float2 buf[];
    const int j = blockIdx.x;
    const int px = d.px, lp = d.lpx;
    float2* zr = Z + (size_t)j * px;
    for (int t = threadIdx.x; t < px; t += blockDim.x) buf[bitrev(t, lp)] = zr[t];
    __syncthreads();
    fft_stages(buf, lp, false, tw, threadIdx.x, blockDim.x);
    for (int t = threadIdx.x; t < px; t += blockDim.x) zr[t] = buf[t];
}

// circulant model: H = 1 / (P(w) + |F[D]|^2 + 1) and, for the initialisation without D, 1 / (P(w) + 1).
// ramp filter: H = 1 / (K / |w| + 1) for both, K = (pi/4) P(0, pi/4), |w| the wrapped radial frequency
// floored at the first non-zero grid frequency.
__global__ void k_response(SliceDesc d, const float2* __restrict__ Z, float* __restrict__ H,
                           float* __restrict__ Hn, bool ramp) {
    const int64_t n = (int64_t)d.px * d.py;
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    const int k = (int)(e / d.px), l = (int)(e % d.px);
    if (ramp) {
        const double K = fmax((double)Z[d.px / 8].x, 0.0) * (0.25 * M_PI);
        const double wy = 2.0 * M_PI * min(k, d.py - k) / d.py, wx = 2.0 * M_PI * min(l, d.px - l) / d.px;
        const double w = fmax(sqrt(wx * wx + wy * wy), 2.0 * M_PI / max(d.px, d.py));
        const float h = (float)(1.0 / (K / w + 1.0));
        H[e] = h;
        Hn[e] = h;
        return;
    }
    const double wy = 2.0 * M_PI * k / d.py, wx = 2.0 * M_PI * l / d.px;
    const double sy = sin(0.5 * wy), sx = sin(0.5 * wx);
    const double dhat = 4.0 * sy * sy + 4.0 * sx * sx;
    const double phat = fmax((double)Z[e].x, 0.0);
    H[e] = (float)(1.0 / (phat + dhat + 1.0));
    Hn[e] = (float)(1.0 / (phat + 1.0));
}

void launch_psf_to_response(const SliceDesc* d_dev, const SliceDesc& d, const BlockMap& cols_map, int ncols,
                            const float2* psf, float2* Z, float* H, float* H_nograd, const float2* tw, bool ramp,
                            cudaStream_t st) {
    const int64_t n = (int64_t)d.px * d.py;
    k_embed_psf<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(d, psf, Z);
    k_fft_rows_full<<<d.py, 256, sizeof(float2) * d.px, st>>>(d, Z, tw);
    k_fft_cols<<<ncols, 256, sizeof(float2) * kColsSmem, st>>>(d_dev, cols_map, Z, nullptr, 1, 1, tw);
    k_response<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(d, Z, H, H_nograd, ramp);
}

cudaError_t fft_init_attributes() {
    const int cols = (int)(sizeof(float2) * kColsSmem);
    cudaError_t e = cudaFuncSetAttribute(k_fft_cols, cudaFuncAttributeMaxDynamicSharedMemorySize, cols);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_prec_cols<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, cols);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_prec_cols<9>, cudaFuncAttributeMaxDynamicSharedMemorySize, cols);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_prec_cols<10>, cudaFuncAttributeMaxDynamicSharedMemorySize, cols);
    return e;
}

}  // namespace dect
