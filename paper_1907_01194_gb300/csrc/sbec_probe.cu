// Arithmetic peak probe (instrumentation of this library, not a step of the
// method).  The FP64 form of the hot path is bound by the FP64 pipe of the
// GPU rather than by HBM bandwidth, so its roofline needs a measured FP64 rate
// next to the measured copy bandwidth.  sbec_probe_fma_peak runs independent
// chains of fused multiply-adds on every SM and reports the achieved rate.
#include <cuda_runtime.h>

#include "sbec.h"

namespace {

constexpr int kChains = 8;        // independent FMA chains per thread (hide the pipe latency)
constexpr int kThreads = 256;
constexpr int kMaxBlocks = 4096;

// per-block sums of the probe (a fixed array of the library image: the probe
// allocates nothing)
static __device__ double g_probe_out[kMaxBlocks];

// Each thread runs kChains chains a <- a * b + c for `iters` steps.  b is just
// below 1 and c small, so every chain converges to c / (1 - b) and stays finite;
// the per-block sum is stored so that no chain can be optimised away.
template <typename T>
__global__ void __launch_bounds__(kThreads) k_fma_probe(T* out, int iters, T b, T c) {
    T a[kChains];
#pragma unroll
    for (int j = 0; j < kChains; ++j) a[j] = T(threadIdx.x + j) * T(1e-3);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int j = 0; j < kChains; ++j) a[j] = fma(a[j], b, c);
    }
    T s = 0;
#pragma unroll
    for (int j = 0; j < kChains; ++j) s += a[j];
    __shared__ T red[kThreads];
    red[threadIdx.x] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        T t = 0;
        for (int k = 0; k < kThreads; ++k) t += red[k];
        out[blockIdx.x] = t;
    }
}

template <typename T>
int probe(int iters, double* gflops) {
    int dev = 0, sms = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fma_probe<T>, kThreads, 0) != cudaSuccess) {
        cudaGetLastError();
        return SBEC_ERR_CUDA;
    }
    if (per_sm < 1) per_sm = 1;
    int blocks = sms * per_sm;
    if (blocks > kMaxBlocks) blocks = kMaxBlocks;
    T* out = nullptr;
    cudaStream_t s = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int rc = SBEC_OK;
    double best = 0.0;
    void* outp = nullptr;
    if (cudaGetSymbolAddress(&outp, g_probe_out) != cudaSuccess || !outp ||
        cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        rc = SBEC_ERR_CUDA;
    }
    out = static_cast<T*>(outp);
    // one warm-up launch, then the best of three timed launches
    for (int rep = 0; rep < 4 && rc == SBEC_OK; ++rep) {
        cudaEventRecord(e0, s);
        k_fma_probe<T><<<blocks, kThreads, 0, s>>>(out, iters, T(0.9999999), T(1e-7));
        cudaEventRecord(e1, s);
        if (cudaEventSynchronize(e1) != cudaSuccess) { rc = SBEC_ERR_CUDA; break; }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        const double flops = 2.0 * kChains * (double)iters * (double)blocks * kThreads;
        if (rep > 0 && ms > 0.f) {
            const double g = flops / (ms * 1e-3) / 1e9;
            if (g > best) best = g;
        }
    }
    if (rc == SBEC_OK && cudaGetLastError() != cudaSuccess) rc = SBEC_ERR_CUDA;
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (s) cudaStreamDestroy(s);
    cudaGetLastError();
    if (rc == SBEC_OK) *gflops = best;
    return rc;
}

}  // namespace

extern "C" int sbec_probe_fma_peak(int precision, int iters, double* gflops) {
    if (!gflops || iters < 1) return SBEC_ERR_ARG;
    if (precision == SBEC_FP64) return probe<double>(iters, gflops);
    if (precision == SBEC_MIXED) return probe<float>(iters, gflops);
    return SBEC_ERR_ARG;
}
