// gp_probe.cu -- measurement only: sustained lane-operation rates of the
// FP32 pipe (dependent FADD chains) and the special-function unit (ex2 and
// rcp approximations) over every SM, timed with CUDA events.  These give
// the denominators of the ALU roofline of the evaluator: out[0] FADD,
// out[1] ex2, out[2] rcp, out[3] rsqrt, out[4] lg2, out[5] sin (lane
// operations per second), out[6] SM count.  The rcp/rsqrt/lg2/sin chains
// carry one FADD per step, which the FP32 pipe absorbs at its higher rate.
#include "gp_internal.cuh"

namespace gpk {

namespace {
constexpr int kChains = 8;
constexpr int kIters = 4096;
constexpr int kBlock = 256;

__global__ void __launch_bounds__(kBlock) fadd_probe(float *sink, float d) {
    float x[kChains];
#pragma unroll
    for (int i = 0; i < kChains; ++i) x[i] = (float)(threadIdx.x + i);
    for (int it = 0; it < kIters; ++it) {
#pragma unroll
        for (int i = 0; i < kChains; ++i) x[i] = __fadd_rn(x[i], d);
    }
    float s = 0.0f;
#pragma unroll
    for (int i = 0; i < kChains; ++i) s += x[i];
    sink[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// chains start from runtime values so that nothing can be folded at compile time
__global__ void __launch_bounds__(kBlock) ex2_probe(float *sink, float d) {
    float x[kChains];
#pragma unroll
    for (int i = 0; i < kChains; ++i) x[i] = d * (float)(threadIdx.x + 3 * i + 1);
    for (int it = 0; it < kIters; ++it) {
#pragma unroll
        for (int i = 0; i < kChains; ++i) {
            float y;
            asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(-x[i]));
            x[i] = y;
        }
    }
    float s = 0.0f;
#pragma unroll
    for (int i = 0; i < kChains; ++i) s += x[i];
    sink[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// x <- mufu(x) + d: one MUFU and one FADD per step; the FADD keeps an
// involution (rcp(rcp(x))) from cancelling and the chain bounded
template <int KIND>
__global__ void __launch_bounds__(kBlock) mufu_probe(float *sink, float d) {
    float x[kChains];
#pragma unroll
    for (int i = 0; i < kChains; ++i) x[i] = 1.0f + d * (float)(threadIdx.x + 3 * i + 1);
    for (int it = 0; it < kIters; ++it) {
#pragma unroll
        for (int i = 0; i < kChains; ++i) {
            float y;
            if (KIND == 0) asm volatile("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x[i]));
            if (KIND == 1) asm volatile("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x[i]));
            if (KIND == 2) asm volatile("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x[i]));
            if (KIND == 3) asm volatile("sin.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x[i]));
            x[i] = __fadd_rn(y, d + 1.0f);
        }
    }
    float s = 0.0f;
#pragma unroll
    for (int i = 0; i < kChains; ++i) s += x[i];
    sink[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <typename F>
cudaError_t time_it(F launch, cudaStream_t st, double *ms) {
    cudaEvent_t a, b;
    cudaError_t e = cudaEventCreate(&a);
    if (e != cudaSuccess) return e;
    e = cudaEventCreate(&b);
    if (e != cudaSuccess) return e;
    launch();  // warm-up
    cudaEventRecord(a, st);
    for (int r = 0; r < 3; ++r) launch();
    cudaEventRecord(b, st);
    e = cudaEventSynchronize(b);
    float f = 0.0f;
    cudaEventElapsedTime(&f, a, b);
    *ms = f / 3.0;
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}
}  // namespace

cudaError_t probe_pipes(double *out, cudaStream_t st) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    float *sink = nullptr;
    const int grid = sms * 8;
    cudaError_t e = cudaMalloc(&sink, sizeof(float) * grid * kBlock);
    if (e != cudaSuccess) return e;
    const double lane_ops = (double)grid * kBlock * kIters * kChains;
    double ms = 0.0;
    e = time_it([&] { fadd_probe<<<grid, kBlock, 0, st>>>(sink, 1e-7f); }, st, &ms);
    if (e == cudaSuccess) out[0] = lane_ops / (ms * 1e-3);
    if (e == cudaSuccess) e = time_it([&] { ex2_probe<<<grid, kBlock, 0, st>>>(sink, 1e-3f); }, st, &ms);
    if (e == cudaSuccess) out[1] = lane_ops / (ms * 1e-3);
    if (e == cudaSuccess) e = time_it([&] { mufu_probe<0><<<grid, kBlock, 0, st>>>(sink, 1e-3f); }, st, &ms);
    if (e == cudaSuccess) out[2] = lane_ops / (ms * 1e-3);
    if (e == cudaSuccess) e = time_it([&] { mufu_probe<1><<<grid, kBlock, 0, st>>>(sink, 1e-3f); }, st, &ms);
    if (e == cudaSuccess) out[3] = lane_ops / (ms * 1e-3);
    if (e == cudaSuccess) e = time_it([&] { mufu_probe<2><<<grid, kBlock, 0, st>>>(sink, 1e-3f); }, st, &ms);
    if (e == cudaSuccess) out[4] = lane_ops / (ms * 1e-3);
    if (e == cudaSuccess) e = time_it([&] { mufu_probe<3><<<grid, kBlock, 0, st>>>(sink, 1e-3f); }, st, &ms);
    if (e == cudaSuccess) out[5] = lane_ops / (ms * 1e-3);
    out[6] = (double)sms;
    out[7] = 0.0;
    cudaFree(sink);
    return e;
}

}  // namespace gpk
