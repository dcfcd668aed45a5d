// Storage formats of the solver's sinogram-domain vectors (a, u^a, R x and the CG sinogram) and of
// the projector's pair textures. Arithmetic is float32 (accumulations, CG scalars) and float64 (the
// decomposition's logs and 2x2 solve) in every format; only loads and stores convert.
//   PREC_F32 : float2 {c, p} per ray, float4 texel {c_lo, p_lo, c_hi, p_hi}
//   PREC_F16 : __half2 per ray, 8-byte texel of two __half2
//   PREC_BF16: __nv_bfloat162 per ray, 8-byte texel of two __nv_bfloat162
// Conversions to the 16-bit formats round to nearest even.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

namespace dect {

// PREC_F64 selects the solver's separate float64 path (solver_f64.cu); the helpers below serve the others
enum { PREC_F32 = 0, PREC_F16 = 1, PREC_BF16 = 2, PREC_F64 = 3 };

struct __align__(8) TexH {
    __half2 lo, hi;
};
struct __align__(8) TexB {
    __nv_bfloat162 lo, hi;
};

struct PrecF32 {
    using S2 = float2;
    using TX = float4;
};
struct PrecF16 {
    using S2 = __half2;
    using TX = TexH;
};
struct PrecBF16 {
    using S2 = __nv_bfloat162;
    using TX = TexB;
};

// read-only loads (through the non-coherent path) and plain loads / stores of a {c, p} pair
__device__ __forceinline__ float2 ldg2(const float2* p) { return __ldg(p); }
__device__ __forceinline__ float2 ldg2(const __half2* p) { return __half22float2(__ldg(p)); }
__device__ __forceinline__ float2 ldg2(const __nv_bfloat162* p) { return __bfloat1622float2(__ldg(p)); }
__device__ __forceinline__ float2 ld2(const float2* p) { return *p; }
__device__ __forceinline__ float2 ld2(const __half2* p) { return __half22float2(*p); }
__device__ __forceinline__ float2 ld2(const __nv_bfloat162* p) { return __bfloat1622float2(*p); }
__device__ __forceinline__ void st2(float2* p, float2 v) { *p = v; }
__device__ __forceinline__ void st2(float* p, float2 v) { *p = v.x; }  // single-channel vectors keep x
__device__ __forceinline__ void st2(__half2* p, float2 v) { *p = __float22half2_rn(v); }
__device__ __forceinline__ void st2(__nv_bfloat162* p, float2 v) { *p = __float22bfloat162_rn(v); }

// pair-texture texels: {c(lo), p(lo), c(hi), p(hi)}; single-channel texels float2 {lo, hi}
__device__ __forceinline__ float4 ldtex(const float4* p) { return __ldg(p); }
__device__ __forceinline__ float4 ldtex(const float2* p) {
    const float2 v = __ldg(p);
    return make_float4(v.x, 0.f, v.y, 0.f);
}
__device__ __forceinline__ float4 ldtex(const TexH* p) {
    const uint2 u = __ldg(reinterpret_cast<const uint2*>(p));
    const float2 a = __half22float2(*reinterpret_cast<const __half2*>(&u.x));
    const float2 b = __half22float2(*reinterpret_cast<const __half2*>(&u.y));
    return make_float4(a.x, a.y, b.x, b.y);
}
__device__ __forceinline__ float4 ldtex(const TexB* p) {
    const uint2 u = __ldg(reinterpret_cast<const uint2*>(p));
    const float2 a = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&u.x));
    const float2 b = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&u.y));
    return make_float4(a.x, a.y, b.x, b.y);
}
__device__ __forceinline__ void sttex(float4* p, float2 lo, float2 hi) { *p = make_float4(lo.x, lo.y, hi.x, hi.y); }
__device__ __forceinline__ void sttex(float2* p, float lo, float hi) { *p = make_float2(lo, hi); }
__device__ __forceinline__ void sttex(TexH* p, float2 lo, float2 hi) {
    TexH t;
    t.lo = __float22half2_rn(lo);
    t.hi = __float22half2_rn(hi);
    *p = t;
}
__device__ __forceinline__ void sttex(TexB* p, float2 lo, float2 hi) {
    TexB t;
    t.lo = __float22bfloat162_rn(lo);
    t.hi = __float22bfloat162_rn(hi);
    *p = t;
}

inline size_t sino_bytes(int prec) { return prec == PREC_F64 ? 16 : (prec == PREC_F32 ? 8 : 4); }
inline size_t texel_bytes(int prec) { return prec == PREC_F64 ? 32 : (prec == PREC_F32 ? 16 : 8); }

}  // namespace dect
