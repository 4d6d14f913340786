// Kernel convolution of the labels without any device allocation.
//
// vesis_surface_weights needs a vesis_system, and creating one allocates
// device memory (cudaMalloc).  Some callers cannot allocate at the moment
// they need the convolution: code that runs while a CUDA stream is being
// captured into a graph (an allocation there breaks or invalidates the
// capture), processes whose device memory is owned by a pool or arena
// that forbids outside allocations, and latency-critical loops that must
// not hit the driver's allocator.  For them this file provides
// vesis_surface_weights_noalloc: the same three integer passes, with the
// two intermediate planes placed in a fixed array in device global memory
// that a device reserves when it loads the library's module (at the first
// call on that device under CUDA's default lazy module loading).
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>
#include <string>

#include "vesis.h"
#include "vesis_internal.cuh"

namespace vesis {
std::string *noalloc_last_error();   // defined in api.cu
}

namespace {

constexpr long long kNoallocMaxCells = VESIS_NOALLOC_MAX_CELLS;
// uint16 pass-1 plane (2 B/cell) followed by the uint32 pass-2 plane
// (4 B/cell, placed at a 256-byte boundary).
constexpr size_t kPlane1Bytes = ((size_t)kNoallocMaxCells * 2 + 255) / 256 * 256;
constexpr size_t kScratchBytes = kPlane1Bytes + (size_t)kNoallocMaxCells * 4;

// Every GPU that loads the library's module holds this array until the
// process exits.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
unsigned char *g_scratch_addr[kMaxDevices] = {nullptr};

int fail(int code, const char *msg)
{
    *vesis::noalloc_last_error() = msg;
    return code;
}

// Device address of the scratch array on the current device (the name
// g_noalloc_scratch is only a host-side stand-in and must not be passed to
// a kernel).  Looked up again on every call whose stream is not being
// captured, so that a module loaded anew (after a device reset, say) is
// seen; while a capture is in progress the address from the last call on
// that device is used.
int scratch_address(cudaStream_t st, unsigned char **out)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return fail(VESIS_E_CUDA, "cudaGetDevice failed");
    if (dev < 0 || dev >= kMaxDevices) return fail(VESIS_E_ARG, "device index out of range");
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cs) != cudaSuccess)
        return fail(VESIS_E_CUDA, "cudaStreamIsCapturing failed");
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (cs == cudaStreamCaptureStatusNone || g_scratch_addr[dev] == nullptr) {
        if (cs != cudaStreamCaptureStatusNone)
            return fail(VESIS_E_ARG,
                        "first call on this device made during a stream capture; "
                        "call once before capturing");
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || p == nullptr)
            return fail(VESIS_E_CUDA, "cudaGetSymbolAddress of the scratch array failed");
        g_scratch_addr[dev] = static_cast<unsigned char *>(p);
    }
    *out = g_scratch_addr[dev];
    return VESIS_OK;
}

}  // namespace

extern "C" int vesis_surface_weights_noalloc(const vesis_params *p, const uint8_t *chi_dev,
                                             uint32_t *W_dev, void *cuda_stream)
{
    using namespace vesis;
    if (!p || !chi_dev || !W_dev) return fail(VESIS_E_ARG, "NULL argument");
    if (p->nx < 1 || p->ny < 1 || p->nz < 1)
        return fail(VESIS_E_ARG, "grid dimensions must be >= 1");
    const long long G = (long long)p->nx * p->ny * p->nz;
    if (G > kNoallocMaxCells)
        return fail(VESIS_E_ARG,
                    "grid larger than VESIS_NOALLOC_MAX_CELLS cells; use vesis_surface_weights");
    if (!(p->h > 0.0)) return fail(VESIS_E_ARG, "h must be > 0");
    if (p->kernel != 0)
        return fail(VESIS_E_ARG, "the no-allocation convolution takes the separable kernel only");
    if (p->trunc_r < 1 || p->trunc_r > kMaxR) return fail(VESIS_E_ARG, "trunc_r must be in 1..8");
    // integer Gaussian weights summing to 256 (same construction as the
    // system's), on the stack
    KernelW kw;
    const double sig = p->gauss_sigma > 0.0 ? p->gauss_sigma : 2.0 * p->h;
    const int r = p->trunc_r;
    double gw[2 * kMaxR + 1];
    double gs = 0.0;
    for (int a = -r; a <= r; ++a) {
        gw[a + r] = std::exp(-(double)(a * a) / (2.0 * (sig / p->h) * (sig / p->h)));
        gs += gw[a + r];
    }
    int qsum = 0;
    kw.r = r;
    for (int a = -r; a <= r; ++a) {
        if (a == 0) continue;
        kw.q[a + r] = (int)std::nearbyint(256.0 * gw[a + r] / gs);
        qsum += kw.q[a + r];
    }
    kw.q[r] = 256 - qsum;
    if (kw.q[r] < 0) return fail(VESIS_E_ARG, "surface kernel weights exceed 256");
    cudaStream_t st = (cudaStream_t)cuda_stream;
    unsigned char *base = nullptr;
    const int rc = scratch_address(st, &base);
    if (rc != VESIS_OK) return rc;
    GridDesc g{};
    g.nx = p->nx;
    g.ny = p->ny;
    g.nz = p->nz;
    g.h = (float)p->h;
    // both planes are written in full before they are read: nothing in the
    // array has to start at zero
    uint16_t *T1 = reinterpret_cast<uint16_t *>(base);
    uint32_t *T2 = reinterpret_cast<uint32_t *>(base + kPlane1Bytes);
    launch_conv_z(g, kw, chi_dev, T1, st);
    launch_conv_y(g, kw, T1, T2, st);
    launch_conv_x(g, kw, T2, W_dev, st);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(VESIS_E_CUDA, cudaGetErrorString(e));
    return VESIS_OK;
}
