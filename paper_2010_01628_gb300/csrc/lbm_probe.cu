// lbm_probe.cu -- arithmetic-throughput probe used as the denominator of the
// FP64 step's ALU roofline: independent FMA chains (8 per thread), one store
// per thread, timed with CUDA events.  Also the self-test of the bounded
// mbarrier wait that the TMA-staged kernels use.
#include <cuda_runtime.h>

#include "lbm_device.cuh"
#include "lbm_internal.h"

namespace {

template <typename T>
__global__ void fma_chains(T* out, int iters, T a, T b) {
    T x0 = (T)threadIdx.x * (T)1e-3, x1 = x0 + 1, x2 = x0 + 2, x3 = x0 + 3, x4 = x0 + 4, x5 = x0 + 5, x6 = x0 + 6,
      x7 = x0 + 7;
    for (int i = 0; i < iters; ++i) {
        x0 = fma(x0, a, b);
        x1 = fma(x1, a, b);
        x2 = fma(x2, a, b);
        x3 = fma(x3, a, b);
        x4 = fma(x4, a, b);
        x5 = fma(x5, a, b);
        x6 = fma(x6, a, b);
        x7 = fma(x7, a, b);
    }
    out[blockIdx.x * blockDim.x + threadIdx.x] = x0 + x1 + x2 + x3 + x4 + x5 + x6 + x7;
}

template <typename T>
cudaError_t rate(int iters, double* fma_per_s) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int blocks = sms * 8, threads = 256;
    T* out = nullptr;
    cudaError_t e = cudaMalloc(&out, (size_t)blocks * threads * sizeof(T));
    if (e != cudaSuccess) return e;
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    float best = 1e30f;
    for (int rep = 0; rep < 3 && e == cudaSuccess; ++rep) {
        cudaEventRecord(a);
        fma_chains<T><<<blocks, threads>>>(out, iters, (T)0.999999, (T)1e-7);
        cudaEventRecord(b);
        e = cudaEventSynchronize(b);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
        if (ms < best) best = ms;
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    cudaFree(out);
    if (e == cudaSuccess) *fma_per_s = (double)blocks * threads * iters * 8.0 / (best * 1e-3);
    return e;
}

// One thread waits (bounded) for phase 0 of an mbarrier expecting one arrival;
// with `arrive` it arrives first and the wait must succeed at once, without it
// nothing completes the phase and the wait must give up after limit_ns.
__global__ void mbar_selftest_kernel(unsigned long long limit_ns, int arrive, int* __restrict__ status) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x != 0) return;
    lbm::mbar_init(&bar, 1);
    lbm::fence_barrier_init();
    if (arrive) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(lbm::smem_u32(&bar)) : "memory");
    *status = lbm::mbar_wait_bounded(&bar, 0, limit_ns) ? (int)LBM_OK : (int)LBM_ERR_TIMEOUT;
}

}  // namespace

extern "C" lbm_status lbm_mbarrier_selftest(double timeout_s, int arrive, int* observed) {
    if (!observed || !(timeout_s > 0.0) || timeout_s > 10.0) return LBM_ERR_ARG;
    int* st = nullptr;
    if (cudaMalloc(&st, sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        return LBM_ERR_OOM;
    }
    cudaError_t e = cudaMemset(st, 0xff, sizeof(int));
    if (e == cudaSuccess) {
        mbar_selftest_kernel<<<1, 32>>>((unsigned long long)(timeout_s * 1e9), arrive ? 1 : 0, st);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    int h = -1;
    if (e == cudaSuccess) e = cudaMemcpy(&h, st, sizeof(int), cudaMemcpyDeviceToHost);
    cudaFree(st);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return LBM_ERR_CUDA;
    }
    *observed = h;
    return LBM_OK;
}

extern "C" lbm_status lbm_probe_fma_rate(double* fp64_fma_per_s, double* fp32_fma_per_s) {
    if (!fp64_fma_per_s || !fp32_fma_per_s) return LBM_ERR_ARG;
    cudaError_t e = rate<double>(1 << 14, fp64_fma_per_s);
    if (e == cudaSuccess) e = rate<float>(1 << 16, fp32_fma_per_s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return LBM_ERR_CUDA;
    }
    return LBM_OK;
}
