// peaks.cu — arithmetic peaks of the current GPU, measured with CUDA events:
// the float64 and float32 fused multiply-add rates.  They are the
// denominators of the arithmetic roofs that the benchmark reports beside the
// HBM roof (the stage's element kernels carry float64 limiter arithmetic on
// GB300's narrow float64 pipe).
#include <cuda_runtime.h>

#include "state.h"

namespace cgl {

// ILP independent FMA chains per thread; a value that is never produced keeps
// every chain live without a store in the timed loop
template <class T, int ILP>
__global__ void __launch_bounds__(256) k_fma_rate(T* out, int iters, T b, T c) {
    T a[ILP];
#pragma unroll
    for (int k = 0; k < ILP; ++k) a[k] = T(threadIdx.x + k) * T(1e-3);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < ILP; ++k) a[k] = fma(a[k], b, c);
    }
    T s = T(0);
#pragma unroll
    for (int k = 0; k < ILP; ++k) s += a[k];
    if (s == T(-1234.5)) out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <class T>
static cgl_status fma_rate(int nsm, T* out, double* flops) {
    constexpr int ILP = 8;
    const int grid = nsm * 8, block = 256;
    // float64: 2 FMA / clock / SM class rates need far fewer iterations
    const int iters = sizeof(T) == 8 ? 2048 : 32768;
    cudaEvent_t a = nullptr, b = nullptr;
    cgl_status rc = CGL_OK;
    if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) {
        rc = set_error(CGL_ECUDA, "cudaEventCreate failed");
    } else {
        k_fma_rate<T, ILP><<<grid, block>>>(out, iters / 8, T(0.999999), T(1e-7));  // warm-up
        float best = 1e30f;
        for (int rep = 0; rep < 3; ++rep) {
            cudaEventRecord(a);
            k_fma_rate<T, ILP><<<grid, block>>>(out, iters, T(0.999999), T(1e-7));
            cudaEventRecord(b);
            cudaError_t e = cudaEventSynchronize(b);
            if (e != cudaSuccess) {
                rc = set_error(CGL_ECUDA, "fma rate kernel: %s", cudaGetErrorString(e));
                break;
            }
            float ms = 0.f;
            cudaEventElapsedTime(&ms, a, b);
            if (ms < best) best = ms;
        }
        if (rc == CGL_OK) *flops = 2.0 * (double)grid * block * ILP * (double)iters / (best * 1e-3);
    }
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
    return rc;
}

}  // namespace cgl

using namespace cgl;

extern "C" cgl_status cgl_measure_peaks(double* fp64_flops, double* fp32_flops) {
    if (!fp64_flops || !fp32_flops) return set_error(CGL_EINVAL, "null argument");
    int dev = 0, nsm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return set_error(CGL_ECUDA, "no usable CUDA device: %s", cudaGetErrorString(e));
    void* out = nullptr;
    e = cudaMalloc(&out, (size_t)nsm * 8 * 256 * sizeof(double));
    if (e != cudaSuccess) return set_error(CGL_EOOM, "cudaMalloc: %s", cudaGetErrorString(e));
    cgl_status rc = fma_rate<double>(nsm, (double*)out, fp64_flops);
    if (rc == CGL_OK) rc = fma_rate<float>(nsm, (float*)out, fp32_flops);
    cudaFree(out);
    return rc;
}
