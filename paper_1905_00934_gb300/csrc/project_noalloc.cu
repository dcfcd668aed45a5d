// dect_project_noalloc: the forward projector for callers that cannot allocate device memory.
//
// dect_project keeps its scratch (the pair textures and the interleaved copy of the image) in
// the geometry handle and allocates it with cudaMalloc on first use. Some callers cannot allow
// that: code running while a CUDA stream is being captured into a graph (cudaMalloc is not a
// stream operation and breaks or invalidates the capture), code whose device memory is handed
// out entirely by its own pool or framework allocator, and fixed-budget deployments that must
// not grow their footprint after start-up. This variant uses a fixed scratch array in device
// global memory instead, defined below at file scope, and calls no allocation routine.
//
// The array is part of the library image: every GPU that loads the library holds it until the
// process exits. Every call uses the same array, so two calls that overlap on the GPU (on
// different streams, or from different host threads) race on it; calls must be ordered. Each call
// rewrites every scratch entry it reads, so nothing from an earlier call needs clearing.
#include <cuda_runtime.h>

#include <mutex>
#include <string>
#include <vector>

#include "dect_internal.cuh"

namespace dect {

// Scratch of the no-allocation projector: TX [nx][ny+3] float4, TY [ny][nx+3] float4 and the
// interleaved image [ny][nx] float2, packed in that order.
static __device__ __align__(256) unsigned char g_noalloc_scratch[DECT_NOALLOC_SCRATCH_BYTES];

// Device address of g_noalloc_scratch per device, looked up once with that device current.
static std::mutex g_noalloc_mu;
static std::vector<unsigned char*> g_noalloc_ptr;

static cudaError_t noalloc_scratch(unsigned char** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if ((int)g_noalloc_ptr.size() <= dev) g_noalloc_ptr.resize(dev + 1, nullptr);
    if (!g_noalloc_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_noalloc_ptr[dev] = static_cast<unsigned char*>(p);
    }
    *out = g_noalloc_ptr[dev];
    return cudaSuccess;
}

size_t noalloc_bytes(int nx, int ny) {
    return sizeof(float4) * ((size_t)nx * (ny + 3) + (size_t)ny * (nx + 3)) + sizeof(float2) * (size_t)nx * ny;
}

}  // namespace dect

struct dect_geom;  // defined in api.cu
namespace dect {
const dect_geom_desc* geom_desc_of(const dect_geom* g);
SliceDesc geom_single_of(const dect_geom* g);
}  // namespace dect

extern "C" dect_status dect_project_noalloc(const dect_geom* g, int32_t nch, const float* x_dev, float* sino_dev,
                                            void* stream) {
    (void)cudaGetLastError();
    if (!g || !x_dev || !sino_dev) {
        dect::set_error("dect_project_noalloc: null argument");
        return DECT_EINVAL;
    }
    if (nch != 1 && nch != 2) {
        dect::set_error("dect_project_noalloc: n_channels must be 1 or 2");
        return DECT_EINVAL;
    }
    const dect_geom_desc* d = dect::geom_desc_of(g);
    const size_t need = dect::noalloc_bytes(d->nx, d->ny);
    if (need > (size_t)DECT_NOALLOC_SCRATCH_BYTES) {
        dect::set_error("dect_project_noalloc: a " + std::to_string(d->nx) + " x " + std::to_string(d->ny) +
                        " image needs " + std::to_string(need) + " bytes of scratch, more than the fixed " +
                        std::to_string((size_t)DECT_NOALLOC_SCRATCH_BYTES) + "; use dect_project");
        return DECT_EINVAL;
    }
    unsigned char* base = nullptr;
    cudaError_t e = dect::noalloc_scratch(&base);
    if (e != cudaSuccess) {
        dect::set_error(std::string("dect_project_noalloc: cudaGetSymbolAddress: ") + cudaGetErrorString(e));
        return DECT_ECUDA;
    }
    float4* tx = reinterpret_cast<float4*>(base);
    float4* ty = tx + (size_t)d->nx * (d->ny + 3);
    float2* img = reinterpret_cast<float2*>(ty + (size_t)d->ny * (d->nx + 3));
    dect::project_single(dect::geom_single_of(g), x_dev, nch, img, tx, ty, sino_dev,
                         reinterpret_cast<cudaStream_t>(stream));
    e = cudaGetLastError();
    if (e != cudaSuccess) {
        dect::set_error(std::string("dect_project_noalloc: ") + cudaGetErrorString(e));
        return DECT_ECUDA;
    }
    return DECT_OK;
}
