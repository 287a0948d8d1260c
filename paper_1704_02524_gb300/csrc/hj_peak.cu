// hj_peak.cu -- FMA-chain microbenchmark: the FP32 FMA rate the device
// sustains, the measured counterpart of the ALU roofline's
// SMs x 128 lanes x 2 flop x clock.
#include <cuda_runtime.h>

#include "hj.h"

namespace {

constexpr int CHAINS = 8;  // independent FMA chains per thread (enough to hide the FMA latency)

// Every thread runs CHAINS independent chains x <- x a + b for `iters`
// rounds (a slightly below 1 keeps the values bounded) and writes one sum,
// so nothing is folded away.  out holds gridDim.x * blockDim.x floats.
__global__ void k_fma_chains(float *out, int iters, float a, float b)
{
    float x[CHAINS];
#pragma unroll
    for (int k = 0; k < CHAINS; ++k) x[k] = 1e-3f * (float)(threadIdx.x + k);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < CHAINS; ++k) x[k] = fmaf(x[k], a, b);
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < CHAINS; ++k) s += x[k];
    out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace

extern "C" hj_status hj_fp32_fma_rate(int device, double *tflops)
{
    if (!tflops) return HJ_EINVAL;
    *tflops = 0.0;
    if (cudaSetDevice(device) != cudaSuccess) return HJ_ECUDA;
    int nsm = 0;
    if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) return HJ_ECUDA;
    const int threads = 256, blocks = nsm * 8, iters = 1 << 16;  // 8 x 256 = 2048 threads per SM
    float *out = nullptr;
    if (cudaMalloc(&out, sizeof(float) * (size_t)blocks * threads) != cudaSuccess) return HJ_ENOMEM;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    hj_status st = HJ_OK;
    float best = 0.f;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) st = HJ_ECUDA;
    for (int rep = 0; st == HJ_OK && rep < 6; ++rep) {  // the first launch warms up
        cudaEventRecord(e0, 0);
        k_fma_chains<<<blocks, threads>>>(out, iters, 0.9999999f, 1e-7f);
        cudaEventRecord(e1, 0);
        if (cudaEventSynchronize(e1) != cudaSuccess || cudaGetLastError() != cudaSuccess) {
            st = HJ_ECUDA;
            break;
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (rep > 0 && ms > 0.f && (best == 0.f || ms < best)) best = ms;
    }
    if (st == HJ_OK && best > 0.f)
        *tflops = 2.0 * CHAINS * (double)iters * blocks * threads / (best * 1e-3) / 1e12;
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(out);
    return st;
}
