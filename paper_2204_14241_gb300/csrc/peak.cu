// Arithmetic peak of the CUDA cores, measured: dependent fused multiply-add chains with enough
// independent chains per thread and threads per SM to keep the FP64 (or FP32) pipe busy. It gives
// the denominator of the FP64-bound kernels' roofline (the FP64 operator passes of the reliable
// updates, the force), which the copy-bandwidth and tensor-core peaks do not cover.
#include "internal.h"

namespace hmc {

constexpr int kPeakChains = 8;

template <typename R>
__global__ void __launch_bounds__(256) k_fma_chain(int iters, R b, R c, R* __restrict__ sink) {
    R a[kPeakChains];
#pragma unroll
    for (int j = 0; j < kPeakChains; ++j) a[j] = (R)(threadIdx.x + j) * (R)1e-3;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int j = 0; j < kPeakChains; ++j) a[j] = fma(a[j], b, c);
    }
    R s = 0;
#pragma unroll
    for (int j = 0; j < kPeakChains; ++j) s += a[j];
    sink[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <typename R>
static int fma_rate(int num_sms, double* out) {
    const int blocks = num_sms * 8, threads = 256;
    const int iters = sizeof(R) == 8 ? 2048 : 65536;
    R* sink = nullptr;
    cudaStream_t st = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int rc = HMC_OK;
    cudaError_t e = cudaMalloc((void**)&sink, (size_t)blocks * threads * sizeof(R));
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    float best = 1e30f;
    for (int rep = 0; rep < 5 && e == cudaSuccess; ++rep) {
        e = cudaEventRecord(e0, st);
        k_fma_chain<R><<<blocks, threads, 0, st>>>(iters, (R)0.999999, (R)1e-7, sink);
        if (e == cudaSuccess) e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaEventRecord(e1, st);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e == cudaSuccess && rep > 0 && ms < best) best = ms;   // the first launch warms up
    }
    if (e != cudaSuccess) rc = cuda_check(nullptr, e, "hmc_fma_peak");
    else *out = 2.0 * kPeakChains * (double)iters * blocks * threads / (best * 1e-3);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (st) cudaStreamDestroy(st);
    if (sink) cudaFree(sink);
    return rc;
}

}  // namespace hmc

extern "C" int hmc_fma_peak(int prec, double* flop_per_s) {
    using namespace hmc;
    if (!flop_per_s || (prec != HMC_FP64 && prec != HMC_FP32)) return fail(nullptr, HMC_ERR_ARG, "hmc_fma_peak: bad argument");
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return cuda_check(nullptr, e, "hmc_fma_peak: device query");
    return prec == HMC_FP64 ? fma_rate<double>(sms, flop_per_s) : fma_rate<float>(sms, flop_per_s);
}
