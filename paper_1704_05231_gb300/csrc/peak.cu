// FP32 CUDA-core throughput probe: the measured denominator of the FP32 bank's roofline.
// Every thread runs 16 independent FMA chains (scalar fmaf, or 8 packed FP32x2 FMAs) for
// `iters` iterations; the results are summed into one store so nothing is optimised away.
#include "internal.h"
#include "conv_fp32.cuh"

namespace gb {

__global__ void __launch_bounds__(256) k_fma_peak(float *out, int iters, int packed, float a, float b)
{
    float acc[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) acc[i] = threadIdx.x * 1e-7f + i;
    if (packed) {
        const float2 a2 = make_float2(a, a), b2 = make_float2(b, b);
        for (int it = 0; it < iters; ++it) {
#pragma unroll
            for (int i = 0; i < 16; i += 2) {
                const float2 r = ffma2(make_float2(acc[i], acc[i + 1]), a2, b2);
                acc[i] = r.x;
                acc[i + 1] = r.y;
            }
        }
    } else {
        for (int it = 0; it < iters; ++it) {
#pragma unroll
            for (int i = 0; i < 16; ++i) acc[i] = fmaf(acc[i], a, b);
        }
    }
    float s = 0.f;
#pragma unroll
    for (int i = 0; i < 16; ++i) s += acc[i];
    if (s == 12345.678f) out[0] = s;   // practically never true; keeps the chains live
}

cudaError_t launch_fma_peak(float *out, int blocks, int iters, int packed, cudaStream_t st)
{
    k_fma_peak<<<blocks, 256, 0, st>>>(out, iters, packed, 0.999999f, 1e-6f);
    return cudaGetLastError();
}

}  // namespace gb
