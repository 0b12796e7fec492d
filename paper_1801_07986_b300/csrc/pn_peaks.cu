// pn_peaks.cu -- pn_measure_peaks: FMA-chain microbenchmarks that give the
// roofline denominators of this library's ALU-bound kernels on the device
// at hand (FP32 FMA, packed FP32x2 FMA, FP64 FMA and single-precision rsqrt
// throughput).
#include <cstdio>

#include "pn_internal.h"

namespace {

constexpr int kChains = 8;       // independent dependency chains per thread
constexpr int kThreads = 256;
constexpr int kBlocksPerSM = 8;

template <typename T>
__global__ void __launch_bounds__(kThreads) k_fma_chain(T *out, int iters, T a, T b)
{
    T acc[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c)
        acc[c] = (T)(1 + c) + (T)threadIdx.x * (T)1e-3;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int c = 0; c < kChains; ++c)
            acc[c] = acc[c] * a + b;
    }
    T s = 0;
#pragma unroll
    for (int c = 0; c < kChains; ++c)
        s += acc[c];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// The same chains on packed pairs of floats: one fma.rn.f32x2 instruction
// (sm_100 family) performs two FP32 FMAs.
__global__ void __launch_bounds__(kThreads) k_fma2_chain(float *out, int iters, float a, float b)
{
    float2 acc[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c)
        acc[c] = make_float2(1.0f + c + threadIdx.x * 1e-3f, 2.0f + c + threadIdx.x * 1e-3f);
    const float2 a2 = make_float2(a, a), b2 = make_float2(b, b);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int c = 0; c < kChains; ++c)
            acc[c] = __ffma2_rn(acc[c], a2, b2);
    }
    float s = 0;
#pragma unroll
    for (int c = 0; c < kChains; ++c)
        s += acc[c].x + acc[c].y;
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void __launch_bounds__(kThreads) k_rsqrt_chain(float *out, int iters)
{
    float acc[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c)
        acc[c] = 1.0f + c + threadIdx.x * 1e-3f;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) {
            float y;
            asm volatile("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(acc[c]));
            acc[c] = y + 1.0f;
        }
    }
    float s = 0;
#pragma unroll
    for (int c = 0; c < kChains; ++c)
        s += acc[c];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <typename F>
double time_ms(cudaStream_t st, F launch, cudaError_t *err)
{
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    launch();   // warm-up
    cudaEventRecord(e0, st);
    launch();
    cudaEventRecord(e1, st);
    *err = cudaEventSynchronize(e1);
    float ms = 0.0f;
    if (*err == cudaSuccess)
        *err = cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return ms;
}

}  // namespace

/*
 * out[0] FP32 FMA TFLOP/s (2 flops per FMA), out[1] FP64 FMA TFLOP/s,
 * out[2] rsqrt.approx.f32 Gop/s, out[3] SM count, out[4] packed FP32x2 FMA
 * TFLOP/s; measured now on `device` with independent FMA chains (every SM
 * busy), timed by CUDA events.
 */
extern "C" pn_status pn_measure_peaks(int device, void *cuda_stream, double out[5])
{
    if (!out)
        return pn::set_error(PN_EINVAL, "pn_measure_peaks: NULL output");
    int prev = -1;
    cudaError_t e = cudaGetDevice(&prev);
    if (e == cudaSuccess && prev != device)
        e = cudaSetDevice(device);
    if (e != cudaSuccess)
        return pn::set_error(PN_ECUDA, "pn_measure_peaks: cudaSetDevice: %s", cudaGetErrorString(e));
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    const int blocks = sms * kBlocksPerSM;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    double *buf = nullptr;
    e = cudaMalloc(&buf, sizeof(double) * blocks * kThreads);
    pn_status status = PN_OK;
    if (e != cudaSuccess) {
        status = pn::set_error(PN_ENOMEM, "pn_measure_peaks: cudaMalloc failed");
    } else {
        const double lanes = (double)blocks * kThreads * kChains;
        const int it32 = 100000, it64 = 2000, itr = 20000;
        cudaError_t err = cudaSuccess;
        const double ms32 = time_ms(st, [&] {
            k_fma_chain<float><<<blocks, kThreads, 0, st>>>((float *)buf, it32, 0.9999f, 1e-7f);
        }, &err);
        const double ms64 = err ? 0.0 : time_ms(st, [&] {
            k_fma_chain<double><<<blocks, kThreads, 0, st>>>(buf, it64, 0.9999, 1e-7);
        }, &err);
        const double msr = err ? 0.0 : time_ms(st, [&] {
            k_rsqrt_chain<<<blocks, kThreads, 0, st>>>((float *)buf, itr);
        }, &err);
        const double ms2 = err ? 0.0 : time_ms(st, [&] {
            k_fma2_chain<<<blocks, kThreads, 0, st>>>((float *)buf, it32 / 2, 0.9999f, 1e-7f);
        }, &err);
        if (err != cudaSuccess) {
            status = pn::set_error(PN_ECUDA, "pn_measure_peaks: %s", cudaGetErrorString(err));
        } else {
            out[0] = 2.0 * lanes * it32 / (ms32 * 1e-3) / 1e12;
            out[1] = 2.0 * lanes * it64 / (ms64 * 1e-3) / 1e12;
            out[2] = lanes * itr / (msr * 1e-3) / 1e9;
            out[3] = sms;
            out[4] = 4.0 * lanes * (it32 / 2) / (ms2 * 1e-3) / 1e12;
        }
        cudaFree(buf);
    }
    if (prev >= 0 && prev != device)
        cudaSetDevice(prev);
    return status;
}
