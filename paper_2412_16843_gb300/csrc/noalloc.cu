// cdi_mass_noalloc: total phase volume sum(phi) * cell_volume of a caller's
// device array, for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc (or any allocating routine): code that
// runs inside a custom allocator or memory-pool callback, programs whose
// device memory is fully reserved up front by another framework, and
// environments that forbid allocation after start-up.  They cannot provide
// the workspace that cdi_mass needs, so this entry point takes only the input
// and output arrays and keeps its scratch (one FP64 partial sum per block) in
// a file-scope __device__ array.  That array is loaded with the library on
// every GPU and stays allocated until the process exits.
//
// The paper has no counterpart: this is an interface convenience, not part
// of the method.
#include "../../include/cdi.h"

#include <cuda_runtime.h>

#include <cstdio>
#include <cstring>
#include <mutex>

namespace {

constexpr int kThreads = 256;
constexpr long long kChunk = 8192;         // elements summed by one block
constexpr int kMaxPartials = 4096;         // scratch capacity (32 KiB)
constexpr long long kMaxElements = kChunk * kMaxPartials;  // 33,554,432
constexpr int kMaxDevices = 64;

// Scratch shared by every call on a device: one partial per block.  It keeps
// the previous call's contents; each call overwrites the partials it reads.
static __device__ __align__(256) double g_noalloc_partials[kMaxPartials];

std::mutex g_setup_mu;
double* g_scratch[kMaxDevices] = {nullptr};

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

__device__ double block_sum(double v) {
    __shared__ double sh[32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    v = warp_sum(v);
    __syncthreads();
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    v = (wid == 0 && lane < (int)((blockDim.x + 31) >> 5)) ? sh[lane] : 0.0;
    if (wid == 0) v = warp_sum(v);
    return v;
}

// block b sums elements [b*kChunk, min((b+1)*kChunk, n)) in a fixed order
__global__ void k_partials(const double* phi, long long n, double* partials) {
    const long long lo = (long long)blockIdx.x * kChunk;
    long long hi = lo + kChunk;
    if (hi > n) hi = n;
    double acc = 0.0;
    for (long long i = lo + threadIdx.x; i < hi; i += blockDim.x) acc += phi[i];
    acc = block_sum(acc);
    if (threadIdx.x == 0) partials[blockIdx.x] = acc;
}

__global__ void k_finish(const double* partials, int nparts, double scale, double* out) {
    double acc = 0.0;
    for (int t = threadIdx.x; t < nparts; t += blockDim.x) acc += partials[t];
    acc = block_sum(acc);
    if (threadIdx.x == 0) *out = acc * scale;
}

void put_err(char* err, size_t len, const char* msg) {
    if (err && len) {
        std::strncpy(err, msg, len - 1);
        err[len - 1] = '\0';
    }
}

}  // namespace

extern "C" cdi_status cdi_mass_noalloc(const double* phi_dev, long long n, double cell_volume, double* mass_dev,
                                       void* cuda_stream, char* err, size_t err_len) {
    put_err(err, err_len, "");
    if (!phi_dev || !mass_dev) {
        put_err(err, err_len, "cdi_mass_noalloc: null input or output pointer");
        return CDI_EINVAL;
    }
    if (n < 1 || n > kMaxElements) {
        char b[160];
        std::snprintf(b, sizeof b, "cdi_mass_noalloc: n = %lld outside [1, %lld] (its fixed scratch holds %d partials)",
                      n, kMaxElements, kMaxPartials);
        put_err(err, err_len, b);
        return CDI_EINVAL;
    }
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        put_err(err, err_len, "cdi_mass_noalloc: no usable current device");
        return CDI_ECUDA;
    }
    double* scratch = nullptr;
    {
        // once per device, with that device current: the device address of the
        // scratch array (in host code its name is only a host-side stand-in).
        // The address is kept for the life of the process, so a device reset
        // (cudaDeviceReset) while the library is loaded is not supported.
        std::lock_guard<std::mutex> lock(g_setup_mu);
        if (!g_scratch[dev]) {
            void* ptr = nullptr;
            e = cudaGetSymbolAddress(&ptr, g_noalloc_partials);
            if (e != cudaSuccess || !ptr) {
                char b[160];
                std::snprintf(b, sizeof b, "cdi_mass_noalloc: cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
                put_err(err, err_len, b);
                return CDI_ECUDA;
            }
            g_scratch[dev] = (double*)ptr;
        }
        scratch = g_scratch[dev];
    }
    // an error left by earlier work would otherwise be reported as this call's launch failure
    e = cudaPeekAtLastError();
    if (e != cudaSuccess) {
        char b[160];
        std::snprintf(b, sizeof b, "cdi_mass_noalloc: a CUDA error from earlier work is pending: %s",
                      cudaGetErrorString(e));
        put_err(err, err_len, b);
        return CDI_ECUDA;
    }
    const int nparts = (int)((n + kChunk - 1) / kChunk);
    cudaStream_t s = (cudaStream_t)cuda_stream;
    k_partials<<<nparts, kThreads, 0, s>>>(phi_dev, n, scratch);
    k_finish<<<1, 1024, 0, s>>>(scratch, nparts, cell_volume, mass_dev);
    e = cudaGetLastError();
    if (e != cudaSuccess) {
        char b[160];
        std::snprintf(b, sizeof b, "cdi_mass_noalloc: launch failed: %s", cudaGetErrorString(e));
        put_err(err, err_len, b);
        return CDI_ECUDA;
    }
    return CDI_OK;
}
