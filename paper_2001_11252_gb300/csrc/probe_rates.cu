// Issue-rate probes of the GPU's arithmetic pipes, the denominators of the
// ALU roofline of the scattering loop (which is bound by instruction issue,
// not by HBM).  Each probe kernel runs independent dependency chains of one
// instruction kind in every thread of a full grid, long enough (tens of
// milliseconds) for clock ramp-up and launch cost to vanish, and the host
// times it with CUDA events.  The rates come out in warp-instructions per
// second for the whole GPU.
#include <cstdint>
#include <cuda_runtime.h>

namespace rg {
namespace {

constexpr int kChains = 8;       // independent chains per thread (hides pipe latency)
constexpr int kUnroll = 16;      // instructions per chain per loop trip

// FP32 fused multiply-add (FMA pipe)
__global__ void __launch_bounds__(256) k_probe_ffma(int trips, float seed, float* sink) {
    float v[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) v[c] = seed + (float)(threadIdx.x + c);
    const float a = 0.999999f, b = 1e-7f;
    for (int t = 0; t < trips; ++t) {
#pragma unroll
        for (int u = 0; u < kUnroll; ++u)
#pragma unroll
            for (int c = 0; c < kChains; ++c) v[c] = __fmaf_rn(v[c], a, b);
    }
    float s = 0.0f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += v[c];
    if (s == 12345.678f) sink[threadIdx.x] = s;   // never true: keeps the chains alive
}

// FP64 fused multiply-add (FP64 pipe)
__global__ void __launch_bounds__(256) k_probe_dfma(int trips, double seed, double* sink) {
    double v[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) v[c] = seed + (double)(threadIdx.x + c);
    const double a = 0.999999999, b = 1e-12;
    for (int t = 0; t < trips; ++t) {
#pragma unroll
        for (int u = 0; u < kUnroll; ++u)
#pragma unroll
            for (int c = 0; c < kChains; ++c) v[c] = __fma_rn(v[c], a, b);
    }
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += v[c];
    if (s == 12345.678) sink[threadIdx.x & 127] = s;
}

// special-function unit: base-2 exponential approximation (MUFU.EX2)
__global__ void __launch_bounds__(256) k_probe_mufu(int trips, float seed, float* sink) {
    float v[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) v[c] = seed * 1e-3f + 1e-4f * (float)c;
    for (int t = 0; t < trips; ++t) {
#pragma unroll
        for (int u = 0; u < kUnroll; ++u)
#pragma unroll
            for (int c = 0; c < kChains; ++c) asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(v[c]) : "f"(-v[c]));
    }
    float s = 0.0f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += v[c];
    if (s == 12345.678f) sink[threadIdx.x] = s;
}

// 32-bit integer multiply-add (IMAD)
__global__ void __launch_bounds__(256) k_probe_imad(int trips, uint32_t seed, uint32_t* sink) {
    uint32_t v[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) v[c] = seed + threadIdx.x * 7u + (uint32_t)c;
    for (int t = 0; t < trips; ++t) {
#pragma unroll
        for (int u = 0; u < kUnroll; ++u)
#pragma unroll
            for (int c = 0; c < kChains; ++c) asm volatile("mad.lo.u32 %0, %0, 1664525, 1013904223;" : "+r"(v[c]));
    }
    uint32_t s = 0u;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s ^= v[c];
    if (s == 0x12345678u) sink[threadIdx.x] = s;
}

template <typename F>
cudaError_t time_probe(F launch, double warp_inst, double& rate) {
    cudaEvent_t e0, e1;
    cudaError_t e = cudaEventCreate(&e0);
    if (e != cudaSuccess) return e;
    e = cudaEventCreate(&e1);
    if (e != cudaSuccess) return e;
    launch();   // warm-up (clocks, module load)
    float best = 0.0f;
    for (int rep = 0; rep < 3 && e == cudaSuccess; ++rep) {
        cudaEventRecord(e0);
        launch();
        cudaEventRecord(e1);
        e = cudaEventSynchronize(e1);
        float ms = 0.0f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e == cudaSuccess && (best == 0.0f || ms < best)) best = ms;
    }
    if (e == cudaSuccess) e = cudaGetLastError();
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    rate = best > 0.0f ? warp_inst / (best * 1e-3) : 0.0;
    return e;
}

}  // namespace

// rates[0..3]: FP32 FMA, FP64 FMA, MUFU EX2, IMAD, in warp-instructions per
// second over the whole device; `scratch` is 4 KiB of device memory that
// the probes write only if a chain lands on an unlikely sentinel value
cudaError_t probe_issue_rates(int sms, void* scratch, double rates[4]) {
    const int block = 256;
    const int grid = sms * 8;   // 2048 threads per SM: every scheduler full
    const double warps = (double)grid * block / 32.0;
    const int trips_f = 32768, trips_d = 512, trips_m = 4096, trips_i = 16384;
    const double per = (double)kChains * kUnroll;
    cudaError_t e;
    e = time_probe([&] { k_probe_ffma<<<grid, block>>>(trips_f, 1.0f, (float*)scratch); }, warps * per * trips_f,
                   rates[0]);
    if (e != cudaSuccess) return e;
    e = time_probe([&] { k_probe_dfma<<<grid, block>>>(trips_d, 1.0, (double*)scratch); }, warps * per * trips_d,
                   rates[1]);
    if (e != cudaSuccess) return e;
    e = time_probe([&] { k_probe_mufu<<<grid, block>>>(trips_m, 1.0f, (float*)scratch); }, warps * per * trips_m,
                   rates[2]);
    if (e != cudaSuccess) return e;
    e = time_probe([&] { k_probe_imad<<<grid, block>>>(trips_i, 1u, (uint32_t*)scratch); }, warps * per * trips_i,
                   rates[3]);
    return e;
}

}  // namespace rg
