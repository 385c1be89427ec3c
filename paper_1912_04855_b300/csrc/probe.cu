// probe.cu -- measured arithmetic peaks of the GPU the library runs on.
//
// The step's kernels are bound by arithmetic and instruction issue, not by
// memory, so their roofline needs the rate at which this GPU retires
// floating-point fused multiply-adds.  Each probe kernel runs independent
// multiply-add chains in every thread of a grid that fills the device (8
// blocks of 256 threads per SM) and is timed with CUDA events: FP32 FFMA,
// FP32 packed two-lane FMA (fma.rn.f32x2, a Blackwell instruction) and FP64
// DFMA.  A multiply-add counts 2 flops.
#include <cuda_runtime.h>

#include "../../include/cspht_probe.h"

namespace {

constexpr int PROBE_THREADS = 256;
constexpr int CHAINS = 8;   // independent chains per thread (hides the FMA latency)
constexpr int UNROLL = 8;   // multiply-adds per chain per loop trip

template <typename T>
__global__ void __launch_bounds__(PROBE_THREADS) k_probe_fma(T *out, T a, T b, int trips) {
    T x[CHAINS];
#pragma unroll
    for (int c = 0; c < CHAINS; ++c) x[c] = (T)(threadIdx.x + c) * (T)1e-3;
    for (int i = 0; i < trips; ++i) {
#pragma unroll
        for (int u = 0; u < UNROLL; ++u)
#pragma unroll
            for (int c = 0; c < CHAINS; ++c) x[c] = fma(x[c], a, b);
    }
    T s = 0;
#pragma unroll
    for (int c = 0; c < CHAINS; ++c) s += x[c];
    if (s == (T)-1) out[blockIdx.x] = s;  // never true for these inputs; keeps the chains live
}

// Two FP32 lanes per instruction: x = x * a + b on packed pairs.
__global__ void __launch_bounds__(PROBE_THREADS) k_probe_fma_f32x2(float *out, float a, float b, int trips) {
    unsigned long long x[CHAINS], a2, b2;
    {
        const unsigned int ua = __float_as_uint(a), ub = __float_as_uint(b);
        a2 = ((unsigned long long)ua << 32) | ua;
        b2 = ((unsigned long long)ub << 32) | ub;
    }
#pragma unroll
    for (int c = 0; c < CHAINS; ++c) {
        const unsigned int lo = __float_as_uint((float)(threadIdx.x + c) * 1e-3f),
                           hi = __float_as_uint((float)(threadIdx.x + c + 1) * 1e-3f);
        x[c] = ((unsigned long long)hi << 32) | lo;
    }
    for (int i = 0; i < trips; ++i) {
#pragma unroll
        for (int u = 0; u < UNROLL; ++u)
#pragma unroll
            for (int c = 0; c < CHAINS; ++c) asm("fma.rn.f32x2 %0, %0, %1, %2;" : "+l"(x[c]) : "l"(a2), "l"(b2));
    }
    float s = 0.0f;
#pragma unroll
    for (int c = 0; c < CHAINS; ++c) s += __uint_as_float((unsigned int)x[c]) + __uint_as_float((unsigned int)(x[c] >> 32));
    if (s == -1.0f) out[blockIdx.x] = s;
}

}  // namespace

extern "C" int cspht_probe_fma(int kind, int trips, double *tflops, double *ms_out) {
    if (kind < CSPHT_PROBE_FP32 || kind > CSPHT_PROBE_FP64 || trips < 1 || !tflops) return -1;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        return -3;
    }
    const int blocks = sms * 8;
    void *out = nullptr;  // written only if a chain hits -1, which these inputs never do
    cudaStream_t st = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int rc = 0;
    if (cudaMalloc(&out, sizeof(double) * blocks) != cudaSuccess || cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        rc = -2;
    } else {
        auto launch = [&](int t) {
            if (kind == CSPHT_PROBE_FP32)
                k_probe_fma<float><<<blocks, PROBE_THREADS, 0, st>>>((float *)out, 0.999f, 1e-4f, t);
            else if (kind == CSPHT_PROBE_FP32X2)
                k_probe_fma_f32x2<<<blocks, PROBE_THREADS, 0, st>>>((float *)out, 0.999f, 1e-4f, t);
            else
                k_probe_fma<double><<<blocks, PROBE_THREADS, 0, st>>>((double *)out, 0.999, 1e-4, t);
        };
        launch(trips / 16 > 0 ? trips / 16 : 1);  // warm-up
        cudaEventRecord(e0, st);
        launch(trips);
        cudaEventRecord(e1, st);
        float ms = 0.0f;
        if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess || !(ms > 0.0f)) {
            rc = -3;
        } else {
            const double lanes = kind == CSPHT_PROBE_FP32X2 ? 2.0 : 1.0;
            const double flops = 2.0 * lanes * CHAINS * UNROLL * (double)trips * PROBE_THREADS * blocks;
            *tflops = flops / (ms * 1e-3) / 1e12;
            if (ms_out) *ms_out = ms;
        }
    }
    cudaGetLastError();
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (st) cudaStreamDestroy(st);
    if (out) cudaFree(out);
    return rc;
}
