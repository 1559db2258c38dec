// probe.cu -- FP64 FMA throughput of the device (roofline denominator).
#include <cuda_runtime.h>

#include "../../include/fockdiag.h"
#include "../../include/fockdiag_probe.h"

namespace {

constexpr int kThreads = 256;
constexpr int kBlocksPerSM = 4;

__global__ void fma_chains(double *out, int iters, double a, double b)
{
    // eight independent chains per thread keep the FP64 pipe saturated
    double x0 = threadIdx.x * 1e-3, x1 = x0 + 1.0, x2 = x0 + 2.0, x3 = x0 + 3.0;
    double x4 = x0 + 4.0, x5 = x0 + 5.0, x6 = x0 + 6.0, x7 = x0 + 7.0;
    for (int i = 0; i < iters; ++i) {
        x0 = fma(x0, a, b); x1 = fma(x1, a, b); x2 = fma(x2, a, b); x3 = fma(x3, a, b);
        x4 = fma(x4, a, b); x5 = fma(x5, a, b); x6 = fma(x6, a, b); x7 = fma(x7, a, b);
    }
    const double r = x0 + x1 + x2 + x3 + x4 + x5 + x6 + x7;
    if (r == -1.0) out[0] = r;   // never true for these inputs; keeps the chains live
}

}  // namespace

extern "C" int fk_measure_fp64_fma_rate(void *ws, size_t ws_bytes, double *tflops, void *stream)
{
    if (!ws || !tflops || ((size_t)ws % 256) != 0) return FK_EWORKSPACE;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return FK_ECUDA;
    const int blocks = sms * kBlocksPerSM;
    if (ws_bytes < 256) return FK_EWORKSPACE;
    cudaStream_t st = (cudaStream_t)stream;
    const int iters = 1 << 14;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return FK_ECUDA;
    if (cudaEventCreate(&e1) != cudaSuccess) { cudaEventDestroy(e0); return FK_ECUDA; }
    fma_chains<<<blocks, kThreads, 0, st>>>((double *)ws, 64, 0.999, 1e-3);
    float best = 1e30f;
    for (int rep = 0; rep < 3; ++rep) {
        cudaEventRecord(e0, st);
        fma_chains<<<blocks, kThreads, 0, st>>>((double *)ws, iters, 0.999, 1e-3);
        cudaEventRecord(e1, st);
        if (cudaEventSynchronize(e1) != cudaSuccess) break;
        float ms = 0;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best) best = ms;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (cudaGetLastError() != cudaSuccess || best >= 1e29f) return FK_ECUDA;
    const double flops = 2.0 * 8.0 * (double)iters * blocks * kThreads;
    *tflops = flops / (best * 1e-3) / 1e12;
    return FK_OK;
}
