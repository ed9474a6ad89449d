// noalloc.cu -- pic_field_energy_noalloc: the field-energy reduction of
// pic_diagnostics for callers that must not allocate device memory.
//
// The two-stage reduction needs scratch for its per-block partial sums.  Here
// that scratch is a file-scope static device array of fixed size, so the
// call allocates nothing: every GPU that loads libpic holds the array
// (NOALLOC_MAX_BLOCKS x PIC_NOALLOC_MAX_COMPONENTS doubles = 64 KB) until the
// process exits.  All calls on a device share it: each call overwrites every
// partial it later reads, so nothing has to be cleared between calls, but
// calls whose work overlaps on the GPU (different streams, no ordering) race
// on the array and give wrong sums.
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/pic.h"

extern "C" void pic_internal_set_global_error(const char* msg);

namespace {

constexpr int NOALLOC_MAX_BLOCKS = 1024;
constexpr int NOALLOC_THREADS = 256;
constexpr int NOALLOC_MAX_DEVICES = 64;

static __device__ __align__(256) double g_noalloc_partials[NOALLOC_MAX_BLOCKS * PIC_NOALLOC_MAX_COMPONENTS];

// Per-device address of g_noalloc_partials (host code may not take the
// address of a __device__ variable directly: its name is a host stand-in).
std::mutex g_mutex;
double* g_partials_ptr[NOALLOC_MAX_DEVICES] = {};

template <class T>
__global__ void sumsq_partials_static(const T* __restrict__ f, long long n, int ncomp, double* __restrict__ partial) {
    __shared__ double red[PIC_NOALLOC_MAX_COMPONENTS][NOALLOC_THREADS / 32];
    for (int c = 0; c < ncomp; ++c) {
        double acc = 0.0;
        const T* fc = f + (long long)c * n;
        for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x) {
            const double v = (double)fc[q];
            acc += v * v;
        }
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
        if ((threadIdx.x & 31) == 0) red[c][threadIdx.x >> 5] = acc;
    }
    __syncthreads();
    if (threadIdx.x < ncomp) {
        double s = 0.0;
        for (int w = 0; w < NOALLOC_THREADS / 32; ++w) s += red[threadIdx.x][w];
        partial[blockIdx.x * ncomp + threadIdx.x] = s;
    }
}

__global__ void sum_partials_static(const double* __restrict__ partial, int nblocks, int ncomp, double scale,
                                    double* __restrict__ out) {
    const int c = threadIdx.x;
    if (c >= ncomp) return;
    double s = 0.0;
    for (int b = 0; b < nblocks; ++b) s += partial[b * ncomp + c];
    out[c] = s * scale;
}

// Device address of the scratch array on the current device `dev`, looked up
// once per device (the lookup also loads this file's module there).
cudaError_t partials_of(int dev, double** out) {
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_partials_ptr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_partials);
        if (e != cudaSuccess || !p) return e != cudaSuccess ? e : cudaErrorInvalidSymbol;
        g_partials_ptr[dev] = static_cast<double*>(p);
    }
    *out = g_partials_ptr[dev];
    return cudaSuccess;
}

}  // namespace

// Set-up of the allocation-free entry point on the current device ahead of
// its first call: the scratch address and both precisions' kernels.  CUDA
// loads modules lazily, so without this the first call (or the first call of
// the other precision) maps the 64 KB array and the kernel code then.
extern "C" int pic_internal_noalloc_preload(void) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= NOALLOC_MAX_DEVICES) return 1;
    double* p = nullptr;
    if (partials_of(dev, &p) != cudaSuccess) return 1;
    cudaFuncAttributes a;
    if (cudaFuncGetAttributes(&a, sumsq_partials_static<float>) != cudaSuccess) return 1;
    if (cudaFuncGetAttributes(&a, sumsq_partials_static<double>) != cudaSuccess) return 1;
    if (cudaFuncGetAttributes(&a, sum_partials_static) != cudaSuccess) return 1;
    return 0;
}

extern "C" pic_status pic_field_energy_noalloc(const void* d_field, int precision, int64_t n, int ncomp, double* d_out,
                                               void* stream) {
    if (!d_field || !d_out || n < 0) {
        pic_internal_set_global_error("pic_field_energy_noalloc: NULL pointer or negative length");
        return PIC_ERR_ARG;
    }
    if (precision != PIC_FP32 && precision != PIC_FP64) {
        pic_internal_set_global_error("pic_field_energy_noalloc: precision must be PIC_FP32 or PIC_FP64");
        return PIC_ERR_ARG;
    }
    if (ncomp < 1 || ncomp > PIC_NOALLOC_MAX_COMPONENTS) {
        pic_internal_set_global_error(
            "pic_field_energy_noalloc: ncomp must be 1..PIC_NOALLOC_MAX_COMPONENTS (8): the static scratch holds "
            "1024 partial sums per component for at most 8 components");
        return PIC_ERR_ARG;
    }
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= NOALLOC_MAX_DEVICES) {
        pic_internal_set_global_error("pic_field_energy_noalloc: no usable current CUDA device");
        return PIC_ERR_CUDA;
    }
    double* partial = nullptr;
    // one-time set-up per device, with that device current
    if (partials_of(dev, &partial) != cudaSuccess) {
        pic_internal_set_global_error("pic_field_energy_noalloc: cudaGetSymbolAddress of the scratch failed");
        return PIC_ERR_CUDA;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    long long want = (n + NOALLOC_THREADS - 1) / NOALLOC_THREADS;
    const int nblocks = (int)(want < 1 ? 1 : (want > NOALLOC_MAX_BLOCKS ? NOALLOC_MAX_BLOCKS : want));
    if (precision == PIC_FP64)
        sumsq_partials_static<double><<<nblocks, NOALLOC_THREADS, 0, s>>>(static_cast<const double*>(d_field), n, ncomp, partial);
    else
        sumsq_partials_static<float><<<nblocks, NOALLOC_THREADS, 0, s>>>(static_cast<const float*>(d_field), n, ncomp, partial);
    sum_partials_static<<<1, 32, 0, s>>>(partial, nblocks, ncomp, 1.0 / 25.132741228718345, d_out);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        pic_internal_set_global_error(cudaGetErrorString(e));
        return PIC_ERR_CUDA;
    }
    return PIC_OK;
}
