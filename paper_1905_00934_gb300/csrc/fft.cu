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
// The FFTs are radix-2 decimation in time in shared memory with a float32
// twiddle table computed once in float64 on the host.
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

// Column group of k_fft_cols on the register path: 8 columns, warp c owns column c (blockDim 256).
// buf holds the group's columns in bit-reversed order on entry; on return, rows in natural order.
template <int LOG>
__device__ void cols_regs(float2* buf, const float* __restrict__ hs, int px, int k0,
                          const float2* __restrict__ tw) {
    constexpr int M = 1 << (LOG - 5), py = 1 << LOG, C = 8;
    const int c = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float2* col = buf + c * py;
    float2 v[M];
#pragma unroll
    for (int m = 0; m < M; ++m) v[m] = col[(m << 5) + lane];
    fft_warp_regs<LOG>(v, lane, false, tw);
    if (hs) {
#pragma unroll
        for (int m = 0; m < M; ++m) col[(m << 5) + lane] = v[m];
        __syncthreads();
        for (int e = threadIdx.x; e < C * py; e += blockDim.x) {
            const int cc = e % C, j = e / C;
            const int k = k0 + cc;
            const float h = k < px ? __ldg(hs + (size_t)j * px + k) : 0.f;
            float2& x = buf[cc * py + j];
            x.x *= h;
            x.y *= h;
        }
        __syncthreads();
#pragma unroll
        for (int m = 0; m < M; ++m) v[m] = col[bitrev((m << 5) + lane, LOG)];
        fft_warp_regs<LOG>(v, lane, true, tw);
    }
    // every lane has passed the shuffles above, so all reads of this column are done
#pragma unroll
    for (int m = 0; m < M; ++m) col[(m << 5) + lane] = v[m];
}



// forward row FFTs of the image rows (Compton + i PE), zero-padded to px
__global__ void __launch_bounds__(256) k_prec_rows_fwd(const SliceDesc* __restrict__ dsl, BlockMap map,
                                                       const float2* __restrict__ r, float2* __restrict__ Z,
                                                       const float2* __restrict__ tw) {
    extern __shared__ float2 buf[];
    int j;
    const int s = slice_of(map, blockIdx.x, j);
    const SliceDesc& d = dsl[s];
    const int px = d.px, lp = d.lpx, nx = d.g.nx;
    const float2* row = r + d.img_off + (size_t)j * nx;
    for (int t = threadIdx.x; t < px; t += blockDim.x)
        buf[bitrev(t, lp)] = t < nx ? __ldg(row + t) : make_float2(0.f, 0.f);
    __syncthreads();
    fft_stages(buf, lp, false, tw, threadIdx.x, blockDim.x);
    float2* zr = Z + d.fft_off + (size_t)j * px;
    for (int t = threadIdx.x; t < px; t += blockDim.x) zr[t] = buf[t];
}

// per group of columns: forward column FFT (rows >= rows_in are zero), optional multiplication by H,
// inverse column FFT; writes rows [0, rows_out)
__global__ void __launch_bounds__(256) k_fft_cols(const SliceDesc* __restrict__ dsl, BlockMap map,
                                                  float2* __restrict__ Z, const float* __restrict__ H, int rows_in_all,
                                                  int rows_out_all, const float2* __restrict__ tw) {
    extern __shared__ float2 buf[];
    int g;
    const int s = slice_of(map, blockIdx.x, g);
    const SliceDesc& d = dsl[s];
    const int px = d.px, py = d.py, lp = d.lpy;
    const int C = precond_cols_per_block(py);
    const int k0 = g * C;
    const int rows_in = rows_in_all ? py : d.g.ny;
    const int rows_out = rows_out_all ? py : d.g.ny;
    float2* zs = Z + d.fft_off;
    // load: consecutive threads take consecutive columns of one row
    for (int e = threadIdx.x; e < C * py; e += blockDim.x) {
        const int c = e % C, j = e / C;
        const int k = k0 + c;
        float2 v = make_float2(0.f, 0.f);
        if (j < rows_in && k < px) v = zs[(size_t)j * px + k];
        buf[c * py + bitrev(j, lp)] = v;
    }
    __syncthreads();
    const float* hs = H ? H + d.h_off : nullptr;
    switch (lp) {  // one slice per block, so the branch is uniform
        case 5: cols_regs<5>(buf, hs, px, k0, tw); break;
        case 6: cols_regs<6>(buf, hs, px, k0, tw); break;
        case 7: cols_regs<7>(buf, hs, px, k0, tw); break;
        case 8: cols_regs<8>(buf, hs, px, k0, tw); break;
        case 9: cols_regs<9>(buf, hs, px, k0, tw); break;
        case 10: cols_regs<10>(buf, hs, px, k0, tw); break;
        default: {  // py < 32 or py >= 2048: shared-memory stages, C columns of blockDim/C threads each
            const int lanes = blockDim.x / C;
            const int c = threadIdx.x / lanes, lane = threadIdx.x % lanes;
            fft_stages(buf + c * py, lp, false, tw, lane, lanes);
            if (hs) {
                for (int e = threadIdx.x; e < C * py; e += blockDim.x) {
                    const int cc = e % C, j = e / C;
                    const int k = k0 + cc;
                    const float h = k < px ? __ldg(hs + (size_t)j * px + k) : 0.f;
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
        if (k < px) zs[(size_t)j * px + k] = buf[cc * py + j];
    }
}

// inverse row FFTs, crop to nx, scale by 1/(px*py): s = {Re, Im}; partial <r, s> per channel
__global__ void __launch_bounds__(256) k_prec_rows_inv(const SliceDesc* __restrict__ dsl, BlockMap map,
                                                       const float2* __restrict__ Z, const float2* __restrict__ r,
                                                       float2* __restrict__ s_out, double* __restrict__ partial,
                                                       const float2* __restrict__ tw) {
    extern __shared__ float2 buf[];
    int j;
    const int s = slice_of(map, blockIdx.x, j);
    const SliceDesc& d = dsl[s];
    const int px = d.px, lp = d.lpx, nx = d.g.nx;
    const float2* zr = Z + d.fft_off + (size_t)j * px;
    for (int t = threadIdx.x; t < px; t += blockDim.x) buf[bitrev(t, lp)] = zr[t];
    __syncthreads();
    fft_stages(buf, lp, true, tw, threadIdx.x, blockDim.x);
    const float scale = 1.0f / ((float)px * (float)d.py);
    const size_t row = d.img_off + (size_t)j * nx;
    for (int t = threadIdx.x; t < nx; t += blockDim.x)
        s_out[row + t] = make_float2(buf[t].x * scale, buf[t].y * scale);
    // <r, s> of the row in the order of the register path (lane l takes t = l, l + 32, ..., then a
    // shuffle tree), so a slice gets the same partials whichever row kernel a batch launches
    if (threadIdx.x < 32) {
        double dc = 0.0, dp = 0.0;
        for (int t = threadIdx.x; t < nx; t += 32) {
            const float2 v = make_float2(buf[t].x * scale, buf[t].y * scale);
            const float2 rv = __ldg(r + row + t);
            dc = fma((double)rv.x, (double)v.x, dc);
            dp = fma((double)rv.y, (double)v.y, dp);
        }
        for (int o = 16; o > 0; o >>= 1) {
            dc += __shfl_down_sync(0xffffffffu, dc, o);
            dp += __shfl_down_sync(0xffffffffu, dp, o);
        }
        if (threadIdx.x == 0) {
            partial[2 * (size_t)blockIdx.x] = dc;
            partial[2 * (size_t)blockIdx.x + 1] = dp;
        }
    }
}

// Row passes on the register path (every slice's padded row length in 32..1024): one warp per row,
// blockDim 32, the row staged in shared memory only for the bit-reversal.
template <int LOG>
__device__ void row_fwd_regs(const float2* __restrict__ row, int nx, float2* __restrict__ zr, float2* buf,
                             const float2* __restrict__ tw) {
    constexpr int M = 1 << (LOG - 5), n = 1 << LOG;
    const int lane = threadIdx.x;
    for (int t = lane; t < n; t += 32) buf[bitrev(t, LOG)] = t < nx ? __ldg(row + t) : make_float2(0.f, 0.f);
    __syncwarp();
    float2 v[M];
#pragma unroll
    for (int m = 0; m < M; ++m) v[m] = buf[(m << 5) + lane];
    fft_warp_regs<LOG>(v, lane, false, tw);
#pragma unroll
    for (int m = 0; m < M; ++m) zr[(m << 5) + lane] = v[m];
}

template <int LOG>
__device__ void row_inv_regs(const float2* __restrict__ zr, float2* buf, const float2* __restrict__ tw, float scale,
                             const float2* __restrict__ r, float2* __restrict__ s_out, int nx, double& dc, double& dp) {
    constexpr int M = 1 << (LOG - 5), n = 1 << LOG;
    const int lane = threadIdx.x;
    for (int t = lane; t < n; t += 32) buf[bitrev(t, LOG)] = zr[t];
    __syncwarp();
    float2 v[M];
#pragma unroll
    for (int m = 0; m < M; ++m) v[m] = buf[(m << 5) + lane];
    fft_warp_regs<LOG>(v, lane, true, tw);
#pragma unroll
    for (int m = 0; m < M; ++m) {
        const int t = (m << 5) + lane;
        if (t < nx) {
            const float2 x = make_float2(v[m].x * scale, v[m].y * scale);
            s_out[t] = x;
            const float2 rv = __ldg(r + t);
            dc = fma((double)rv.x, (double)x.x, dc);
            dp = fma((double)rv.y, (double)x.y, dp);
        }
    }
}

__global__ void __launch_bounds__(32) k_prec_rows_fwd_w(const SliceDesc* __restrict__ dsl, BlockMap map,
                                                        const float2* __restrict__ r, float2* __restrict__ Z,
                                                        const float2* __restrict__ tw) {
    extern __shared__ float2 buf[];
    int j;
    const int s = slice_of(map, blockIdx.x, j);
    const SliceDesc& d = dsl[s];
    const float2* row = r + d.img_off + (size_t)j * d.g.nx;
    float2* zr = Z + d.fft_off + (size_t)j * d.px;
    switch (d.lpx) {
        case 5: row_fwd_regs<5>(row, d.g.nx, zr, buf, tw); break;
        case 6: row_fwd_regs<6>(row, d.g.nx, zr, buf, tw); break;
        case 7: row_fwd_regs<7>(row, d.g.nx, zr, buf, tw); break;
        case 8: row_fwd_regs<8>(row, d.g.nx, zr, buf, tw); break;
        case 9: row_fwd_regs<9>(row, d.g.nx, zr, buf, tw); break;
        default: row_fwd_regs<10>(row, d.g.nx, zr, buf, tw); break;
    }
}

__global__ void __launch_bounds__(32) k_prec_rows_inv_w(const SliceDesc* __restrict__ dsl, BlockMap map,
                                                        const float2* __restrict__ Z, const float2* __restrict__ r,
                                                        float2* __restrict__ s_out, double* __restrict__ partial,
                                                        const float2* __restrict__ tw) {
    extern __shared__ float2 buf[];
    int j;
    const int s = slice_of(map, blockIdx.x, j);
    const SliceDesc& d = dsl[s];
    const float2* zr = Z + d.fft_off + (size_t)j * d.px;
    const size_t row = d.img_off + (size_t)j * d.g.nx;
    const float scale = 1.0f / ((float)d.px * (float)d.py);
    double dc = 0.0, dp = 0.0;
    switch (d.lpx) {
        case 5: row_inv_regs<5>(zr, buf, tw, scale, r + row, s_out + row, d.g.nx, dc, dp); break;
        case 6: row_inv_regs<6>(zr, buf, tw, scale, r + row, s_out + row, d.g.nx, dc, dp); break;
        case 7: row_inv_regs<7>(zr, buf, tw, scale, r + row, s_out + row, d.g.nx, dc, dp); break;
        case 8: row_inv_regs<8>(zr, buf, tw, scale, r + row, s_out + row, d.g.nx, dc, dp); break;
        case 9: row_inv_regs<9>(zr, buf, tw, scale, r + row, s_out + row, d.g.nx, dc, dp); break;
        default: row_inv_regs<10>(zr, buf, tw, scale, r + row, s_out + row, d.g.nx, dc, dp); break;
    }
    for (int o = 16; o > 0; o >>= 1) {
        dc += __shfl_down_sync(0xffffffffu, dc, o);
        dp += __shfl_down_sync(0xffffffffu, dp, o);
    }
    if (threadIdx.x == 0) {
        partial[2 * (size_t)blockIdx.x] = dc;
        partial[2 * (size_t)blockIdx.x + 1] = dp;
    }
}

void launch_precond(const SliceDesc* dsl, const BlockMap& rows_map, int nrows_blk, const BlockMap& cols_map,
                    int ncols_blk, const float* H, const float2* r, float2* s, float2* Z, double* partial_rs,
                    const float2* tw, int max_px, int min_px, cudaStream_t st) {
    const bool warp_rows = min_px >= 32 && max_px <= 1024;
    if (warp_rows)
        k_prec_rows_fwd_w<<<nrows_blk, 32, sizeof(float2) * max_px, st>>>(dsl, rows_map, r, Z, tw);
    else
        k_prec_rows_fwd<<<nrows_blk, 256, sizeof(float2) * max_px, st>>>(dsl, rows_map, r, Z, tw);
    // C(py) * py <= 8192 complex entries for every py <= 4096
    k_fft_cols<<<ncols_blk, 256, sizeof(float2) * 8192, st>>>(dsl, cols_map, Z, H, 0, 0, tw);
    if (warp_rows)
        k_prec_rows_inv_w<<<nrows_blk, 32, sizeof(float2) * max_px, st>>>(dsl, rows_map, Z, r, s, partial_rs, tw);
    else
        k_prec_rows_inv<<<nrows_blk, 256, sizeof(float2) * max_px, st>>>(dsl, rows_map, Z, r, s, partial_rs, tw);
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
    k_fft_cols<<<ncols, 256, sizeof(float2) * 8192, st>>>(d_dev, cols_map, Z, nullptr, 1, 1, tw);
    k_response<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(d, Z, H, H_nograd, ramp);
}

cudaError_t fft_init_attributes() {
    return cudaFuncSetAttribute(k_fft_cols, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(sizeof(float2) * 8192));
}

}  // namespace dect
