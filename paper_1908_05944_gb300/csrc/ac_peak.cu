// Measured FMA throughput of the device (FP32 and FP64), the denominator the
// per-atom kernel's arithmetic is compared with: independent FMA chains in
// registers, one launch filling every SM, timed with CUDA events. Not part of
// the method; the bench reports it beside the peak derived from unit counts.
#include "ac_internal.cuh"

namespace ac {

constexpr int PEAK_CHAINS = 8;
constexpr int PEAK_THREADS = 256;

template <class T>
__global__ void __launch_bounds__(PEAK_THREADS) k_fma_peak(T* __restrict__ sink, int iters, T a, T b) {
    T x[PEAK_CHAINS];
#pragma unroll
    for (int c = 0; c < PEAK_CHAINS; c++) x[c] = (T)(threadIdx.x & 7) * (T)0.125 + (T)c;
    for (int i = 0; i < iters; i++) {
#pragma unroll
        for (int c = 0; c < PEAK_CHAINS; c++) x[c] = fma(x[c], a, b);
    }
    T s = 0;
#pragma unroll
    for (int c = 0; c < PEAK_CHAINS; c++) s += x[c];
    if (s == (T)-1) sink[0] = s;  // never true: keeps the chains live
}

template <class T>
static int fma_peak(int iters, cudaStream_t s, double* flops, float* ms_out) {
    int dev = 0, sms = 0, per_sm = 0;
    AC_CUDA(cudaGetDevice(&dev));
    AC_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    AC_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fma_peak<T>, PEAK_THREADS, 0));
    const int blocks = sms * (per_sm > 0 ? per_sm : 1);
    DevBuf sink;
    AC_TRY(sink.reserve(sizeof(T), s));
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    AC_CUDA(cudaEventCreate(&e0));
    AC_CUDA(cudaEventCreate(&e1));
    // one untimed launch, then the timed one
    k_fma_peak<T><<<blocks, PEAK_THREADS, 0, s>>>(sink.as<T>(), iters / 8 > 0 ? iters / 8 : 1, (T)0.9999999,
                                                   (T)1e-7);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaEventRecord(e0, s);
    if (e == cudaSuccess) {
        k_fma_peak<T><<<blocks, PEAK_THREADS, 0, s>>>(sink.as<T>(), iters, (T)0.9999999, (T)1e-7);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaEventRecord(e1, s);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess) return cuda_fail(e, "FMA peak probe", __FILE__, __LINE__);
    *flops = 2.0 * PEAK_CHAINS * (double)iters * (double)blocks * PEAK_THREADS / (ms * 1e-3);
    if (ms_out) *ms_out = ms;
    return AC_OK;
}

}  // namespace ac

using namespace ac;

extern "C" int ac_fma_peak(int fp64, int iters, void* stream, double* flops_per_s, float* ms) {
    if (!flops_per_s || iters < 1) return fail(AC_ERR_INVALID_ARG, "NULL output or iters < 1");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    StreamScope scope(s);
    return fp64 ? fma_peak<double>(iters, s, flops_per_s, ms) : fma_peak<float>(iters, s, flops_per_s, ms);
}
