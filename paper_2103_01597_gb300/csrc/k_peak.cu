// Arithmetic-rate probes: the FMA throughput a kernel of this library reaches
// on the FP64 and FP32 pipes of the device it runs on, measured rather than
// taken from a datasheet, as the denominators of the binary64 substep's
// roofline (its bound is the FP64 pipe, not memory).
//
// Each thread runs CH independent FMA chains x <- x a + b with |a| < 1 (the
// values stay bounded and normal), UNROLL steps per loop iteration; the chains'
// sum is compared with a value it cannot take, so nothing is dead code.  The
// grid is 8 CTAs of 256 threads per SM: enough independent FMAs in flight to
// cover the pipes' latency.
#include "ac_internal.h"

namespace ac {

constexpr int PEAK_CH = 8;
constexpr int PEAK_UNROLL = 16;
constexpr int PEAK_THREADS = 256;

static __device__ double g_peak_sink;

template <typename T>
__global__ void __launch_bounds__(PEAK_THREADS) fma_chain_kernel(int iters, T a, T b) {
    T x[PEAK_CH];
#pragma unroll
    for (int c = 0; c < PEAK_CH; ++c) x[c] = (T)(threadIdx.x + 1 + c) * (T)1e-3;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < PEAK_UNROLL; ++u)
#pragma unroll
            for (int c = 0; c < PEAK_CH; ++c) x[c] = fma(x[c], a, b);
    }
    T s = (T)0;
#pragma unroll
    for (int c = 0; c < PEAK_CH; ++c) s += x[c];
    if (s == (T)-1) g_peak_sink = (double)s;  // never true: the chains stay positive
}

template <typename T>
static cudaError_t fma_rate(int sms, double target_s, double *rate, cudaStream_t st) {
    const int blocks = 8 * sms;
    const double per_iter = (double)blocks * PEAK_THREADS * PEAK_UNROLL * PEAK_CH;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    int iters = 64;
    double best = 0.0;
    for (int round = 0; e == cudaSuccess && round < 8; ++round) {
        fma_chain_kernel<T><<<blocks, PEAK_THREADS, 0, st>>>(iters, (T)0.999999, (T)1e-7);
        e = cudaEventRecord(e0, st);
        if (e != cudaSuccess) break;
        fma_chain_kernel<T><<<blocks, PEAK_THREADS, 0, st>>>(iters, (T)0.999999, (T)1e-7);
        e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaEventRecord(e1, st);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e != cudaSuccess) break;
        const double s = ms * 1e-3;
        if (s > 0.25 * target_s) {
            const double r = per_iter * iters / s;
            best = r > best ? r : best;
        }
        if (s < target_s && iters < (1 << 24)) {  // grow to the target duration
            const double grow = s > 0 ? target_s / s : 16.0;
            iters = (int)(iters * (grow > 16.0 ? 16.0 : (grow < 1.0 ? 1.0 : grow))) + 1;
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    *rate = best;
    return e;
}

}  // namespace ac

extern "C" int ac_diag_fma_rate(int precision, double *fma_per_s, void *stream) {
    if (!fma_per_s || (precision != AC_FP64 && precision != AC_FP32)) return AC_ERR_ARG;
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return ac::ac_report_cuda(e);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    e = precision == AC_FP64 ? ac::fma_rate<double>(sms, 0.05, fma_per_s, st)
                             : ac::fma_rate<float>(sms, 0.05, fma_per_s, st);
    return e == cudaSuccess ? AC_OK : ac::ac_report_cuda(e);
}
