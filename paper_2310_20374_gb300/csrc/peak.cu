// peak.cu -- measured FP32 and FP64 fused multiply-add throughput of the
// device, the denominators of the ALU-bound stages' roofline fractions (the
// near field, M2L and the collision prefilter in FP32; their FP64 forms).
//
// Every thread runs CHAINS independent chains x <- x * a + b for `iters`
// iterations (enough independent work to keep every FMA pipe issuing), then
// writes the sum of its chains to its own slot of an output buffer of
// grid * block elements, so no access leaves the buffer and the compiler
// cannot drop the chains.  FLOPs per launch = 2 * CHAINS * iters * threads.
#include <algorithm>

#include "ctx.h"

namespace ncorp {

constexpr int FMA_CHAINS = 8;
constexpr int FMA_THREADS = 256;

template <typename T>
__global__ void __launch_bounds__(FMA_THREADS) k_fma_chain(T *out, int iters, T a, T b) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    T x[FMA_CHAINS];
#pragma unroll
    for (int k = 0; k < FMA_CHAINS; k++) x[k] = static_cast<T>(t + k) * static_cast<T>(1e-7);
    for (int i = 0; i < iters; i++) {
#pragma unroll
        for (int k = 0; k < FMA_CHAINS; k++) x[k] = fma(x[k], a, b);
    }
    T s = T(0);
#pragma unroll
    for (int k = 0; k < FMA_CHAINS; k++) s += x[k];
    out[t] = s;
}

}  // namespace ncorp

extern "C" int ncorp_fma_peak(int device, int precision, void *cuda_stream, double *flop_per_s) {
    using namespace ncorp;
    if (!flop_per_s || (precision != NCORP_FP64 && precision != NCORP_MIXED)) return NCORP_EINVAL;
    *flop_per_s = 0.0;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    void *buf = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int status = NCORP_OK;
    do {
        int sms = 0;
        if (cudaSetDevice(device) != cudaSuccess ||
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) {
            status = NCORP_ECUDA;
            break;
        }
        const int grid = 8 * sms;   // 64 resident warps per SM
        const bool f64 = precision == NCORP_FP64;
        // about 4 ms (FP32) and 4 ms (FP64) per launch at the measured rates
        const int iters = f64 ? 1 << 10 : 1 << 16;
        const size_t bytes = static_cast<size_t>(grid) * FMA_THREADS * (f64 ? sizeof(double) : sizeof(float));
        if (cudaMalloc(&buf, bytes) != cudaSuccess) {
            status = NCORP_ENOMEM;
            break;
        }
        if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
            status = NCORP_ECUDA;
            break;
        }
        float best = 0.0f;
        for (int rep = 0; rep < 6 && status == NCORP_OK; rep++) {   // the first launch is a warm-up
            if (cudaEventRecord(e0, s) != cudaSuccess) status = NCORP_ECUDA;
            if (f64)
                k_fma_chain<double><<<grid, FMA_THREADS, 0, s>>>(static_cast<double *>(buf), iters, 0.999999, 1e-9);
            else
                k_fma_chain<float><<<grid, FMA_THREADS, 0, s>>>(static_cast<float *>(buf), iters, 0.999999f, 1e-9f);
            if (cudaGetLastError() != cudaSuccess || cudaEventRecord(e1, s) != cudaSuccess ||
                cudaEventSynchronize(e1) != cudaSuccess) {
                status = NCORP_ECUDA;
                break;
            }
            float ms = 0.0f;
            if (cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) status = NCORP_ECUDA;
            if (rep > 0 && ms > 0.0f && (best == 0.0f || ms < best)) best = ms;
        }
        if (status == NCORP_OK && best > 0.0f)
            *flop_per_s = 2.0 * FMA_CHAINS * static_cast<double>(iters) * grid * FMA_THREADS / (best * 1e-3);
    } while (false);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (buf) cudaFree(buf);
    return status;
}
