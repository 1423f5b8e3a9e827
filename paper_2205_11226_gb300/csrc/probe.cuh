// Throughput probes of the two units the concealment kernel leans on: FP32 FMA and the
// MUFU exp2 unit.  Measured rather than taken from a data sheet: they are the
// denominators of the ALU and exp roofline fractions the benchmark reports.
#pragma once

#include <cuda_runtime.h>

namespace sk {

constexpr int kProbeIters = 4096;
constexpr int kProbeChains = 8;  // independent dependency chains per thread

__global__ void __launch_bounds__(256) probe_fma_kernel(float* out, float b, float c) {
    float a[kProbeChains];
#pragma unroll
    for (int q = 0; q < kProbeChains; ++q) a[q] = (float)(threadIdx.x + q);
    for (int it = 0; it < kProbeIters; ++it) {
#pragma unroll
        for (int q = 0; q < kProbeChains; ++q) a[q] = __fmaf_rn(a[q], b, c);
    }
    float s = 0.0f;
#pragma unroll
    for (int q = 0; q < kProbeChains; ++q) s += a[q];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void __launch_bounds__(256) probe_ex2_kernel(float* out, float b) {
    float a[kProbeChains];
#pragma unroll
    for (int q = 0; q < kProbeChains; ++q) a[q] = -1.0f - 1e-3f * (float)(threadIdx.x + q);
    for (int it = 0; it < kProbeIters; ++it) {
#pragma unroll
        for (int q = 0; q < kProbeChains; ++q) {
            float r;
            asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(a[q]));
            a[q] = r * b - 1.0f;  // stays in (-2, -0.5): no overflow, no denormals
        }
    }
    float s = 0.0f;
#pragma unroll
    for (int q = 0; q < kProbeChains; ++q) s += a[q];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace sk
