// Arithmetic peak probes for the roofline denominators of the measurement.
//
// The quadrature and the line solves run on the FP32 (or FP64) FMA pipes, not on tensor
// cores, so their roofline needs the rate of plain fused multiply-adds on this GPU.  Each
// probe launches four 256-thread CTAs per SM; every thread runs CH independent FMA chains
// (a = a * b + c, |b| < 1 so the values stay bounded) for a fixed number of iterations, and
// the kernel's device time (CUDA events on the launching stream, best of three after a
// warm-up) gives flops / s = 2 * chains * iterations * threads / time.  The FP32 probe runs
// the packed form (__ffma2_rn: two FP32 FMAs per instruction) too and reports the faster.
#include <cuda_runtime.h>

#include "wf.h"

namespace {

template <int CH>
__global__ void __launch_bounds__(256) k_peak_f32(float* out, int iters, float b, float c) {
    float a[CH];
#pragma unroll
    for (int i = 0; i < CH; ++i) a[i] = 1e-3f * (threadIdx.x + i);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < 8; ++u)
#pragma unroll
            for (int i = 0; i < CH; ++i) a[i] = fmaf(a[i], b, c);
    }
    float s = 0.f;
#pragma unroll
    for (int i = 0; i < CH; ++i) s += a[i];
    if (s == 1234.5f) out[blockIdx.x] = s;  // keeps the chains live; practically never stored
}

template <int CH>
__global__ void __launch_bounds__(256) k_peak_f32x2(float* out, int iters, float b, float c) {
    float2 a[CH];
    const float2 b2 = make_float2(b, b), c2 = make_float2(c, c);
#pragma unroll
    for (int i = 0; i < CH; ++i) a[i] = make_float2(1e-3f * (threadIdx.x + i), 2e-3f * (threadIdx.x + i));
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < 8; ++u)
#pragma unroll
            for (int i = 0; i < CH; ++i) a[i] = __ffma2_rn(a[i], b2, c2);
    }
    float s = 0.f;
#pragma unroll
    for (int i = 0; i < CH; ++i) s += a[i].x + a[i].y;
    if (s == 1234.5f) out[blockIdx.x] = s;
}

template <int CH>
__global__ void __launch_bounds__(256) k_peak_f64(double* out, int iters, double b, double c) {
    double a[CH];
#pragma unroll
    for (int i = 0; i < CH; ++i) a[i] = 1e-3 * (threadIdx.x + i);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < 8; ++u)
#pragma unroll
            for (int i = 0; i < CH; ++i) a[i] = fma(a[i], b, c);
    }
    double s = 0.0;
#pragma unroll
    for (int i = 0; i < CH; ++i) s += a[i];
    if (s == 1234.5) out[blockIdx.x] = s;
}

// Best-of-three device time (ms) of launch(), after one warm-up launch.
template <typename L>
cudaError_t time_best(L&& launch, cudaStream_t s, float* best) {
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e == cudaSuccess) {
        launch();
        e = cudaGetLastError();
    }
    *best = 1e30f;
    for (int r = 0; r < 3 && e == cudaSuccess; ++r) {
        cudaEventRecord(e0, s);
        launch();
        cudaEventRecord(e1, s);
        e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e == cudaSuccess && ms < *best) *best = ms;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    return e;
}

}  // namespace

extern "C" int wf_measure_fma_peak(int precision, double* tflops) {
    if (!tflops || (precision != WF_FP32 && precision != WF_FP64)) return WF_EINVAL;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return WF_ECUDA;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return WF_ECUDA;
    constexpr int CH = 8, THREADS = 256, PER_SM = 4, UNROLL = 8;
    const int blocks = sms * PER_SM;
    void* out = nullptr;
    if (cudaMalloc(&out, (size_t)blocks * sizeof(double)) != cudaSuccess) return WF_ENOMEM;
    cudaStream_t s = nullptr;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) {
        cudaFree(out);
        return WF_ECUDA;
    }
    const double threads = (double)blocks * THREADS;
    cudaError_t e = cudaSuccess;
    double best = 0.0;
    if (precision == WF_FP32) {
        const int iters = 32768;  // 0.65 Tflop per launch: about 8 ms at the expected rate
        float ms = 0.f;
        e = time_best([&] { k_peak_f32<CH><<<blocks, THREADS, 0, s>>>((float*)out, iters, 0.999f, 1e-3f); }, s, &ms);
        if (e == cudaSuccess) best = 2.0 * CH * UNROLL * (double)iters * threads / (ms * 1e-3) / 1e12;
        if (e == cudaSuccess) {
            e = time_best([&] { k_peak_f32x2<CH><<<blocks, THREADS, 0, s>>>((float*)out, iters / 2, 0.999f, 1e-3f); },
                          s, &ms);
            // two FP32 FMAs per packed instruction
            const double t2 = 2.0 * 2 * CH * UNROLL * (double)(iters / 2) * threads / (ms * 1e-3) / 1e12;
            if (e == cudaSuccess && t2 > best) best = t2;
        }
    } else {
        const int iters = 512;  // 10 Gflop: about 8 ms at the expected FP64 rate
        float ms = 0.f;
        e = time_best([&] { k_peak_f64<CH><<<blocks, THREADS, 0, s>>>((double*)out, iters, 0.999, 1e-3); }, s, &ms);
        if (e == cudaSuccess) best = 2.0 * CH * UNROLL * (double)iters * threads / (ms * 1e-3) / 1e12;
    }
    cudaStreamDestroy(s);
    cudaFree(out);
    if (e != cudaSuccess) return WF_ECUDA;
    *tflops = best;
    return WF_OK;
}

// Host-link probe: the copy rate between caller-owned pinned host arrays and the device, alone in
// each direction and with both directions at once (two streams), each best of three after a
// warm-up.  It bounds any end-to-end step whose inputs arrive from, and whose results return to,
// host memory.
extern "C" int wf_measure_host_link(const void* host_in, void* host_out, size_t bytes, double* gbs_h2d,
                                    double* gbs_d2h, double* gbs_both) {
    if (!host_in || !host_out || bytes == 0 || !gbs_h2d || !gbs_d2h || !gbs_both) return WF_EINVAL;
    void *din = nullptr, *dout = nullptr;
    if (cudaMalloc(&din, bytes) != cudaSuccess) return WF_ENOMEM;
    if (cudaMalloc(&dout, bytes) != cudaSuccess) {
        cudaFree(din);
        return WF_ENOMEM;
    }
    cudaStream_t s = nullptr, s2 = nullptr;
    cudaEvent_t fork = nullptr, join = nullptr;
    cudaError_t e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s2, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&fork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&join, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaMemsetAsync(dout, 0, bytes, s);
    float t_in = 0.f, t_out = 0.f, t_both = 0.f;
    if (e == cudaSuccess)
        e = time_best([&] { cudaMemcpyAsync(din, host_in, bytes, cudaMemcpyHostToDevice, s); }, s, &t_in);
    if (e == cudaSuccess)
        e = time_best([&] { cudaMemcpyAsync(host_out, dout, bytes, cudaMemcpyDeviceToHost, s); }, s, &t_out);
    if (e == cudaSuccess)
        e = time_best(
            [&] {
                cudaEventRecord(fork, s);
                cudaStreamWaitEvent(s2, fork, 0);
                cudaMemcpyAsync(din, host_in, bytes, cudaMemcpyHostToDevice, s);
                cudaMemcpyAsync(host_out, dout, bytes, cudaMemcpyDeviceToHost, s2);
                cudaEventRecord(join, s2);
                cudaStreamWaitEvent(s, join, 0);
            },
            s, &t_both);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (join) cudaEventDestroy(join);
    if (fork) cudaEventDestroy(fork);
    if (s2) cudaStreamDestroy(s2);
    if (s) cudaStreamDestroy(s);
    cudaFree(dout);
    cudaFree(din);
    if (e != cudaSuccess) return WF_ECUDA;
    *gbs_h2d = (double)bytes / (t_in * 1e-3) / 1e9;
    *gbs_d2h = (double)bytes / (t_out * 1e-3) / 1e9;
    *gbs_both = 2.0 * (double)bytes / (t_both * 1e-3) / 1e9;
    return WF_OK;
}
