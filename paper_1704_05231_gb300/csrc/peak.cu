// Measurement probes.
//   k_fma_peak       FP32 CUDA-core throughput, the measured denominator of the FP32 bank's
//                    roofline: every thread runs 16 independent FMA chains (scalar fmaf, or 8
//                    packed FP32x2 FMAs) for `iters` iterations; the results are summed into one
//                    store so nothing is optimised away.
//   k_store_pattern  the output stream of the tensor-core SDFT without its arithmetic: the same
//                    CTA shape (16 storing warps, one CTA per SM), tile order (128 pixels of one
//                    row per tile, tiles t = CTA + i * grid) and per-warp plane ranges, writing
//                    non-zero values (a zero fill is faster through the memory's zero
//                    compression), so that its bandwidth is the ceiling of that store pattern.
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

// warp w: pixels 32 (w % 4) .. + 31 of the tile, planes [g nplanes / 4, (g + 1) nplanes / 4) with
// g = w / 4; one complex64 store per pixel and plane, 32 consecutive pixels per instruction.
__global__ void __launch_bounds__(512, 1) k_store_pattern(float2 *out, int64_t nplanes, int H, int W)
{
    const int warp = (int)(threadIdx.x >> 5), lane = (int)(threadIdx.x & 31);
    const int q = warp & 3, g = warp >> 2;
    const int tiles_x = W / 128;
    const int64_t plane = (int64_t)H * W;
    const int64_t p0 = g * nplanes / 4, p1 = (g + 1) * nplanes / 4;
    const int ntiles = tiles_x * H;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const int y = t / tiles_x, x = (t % tiles_x) * 128 + 32 * q + lane;
        float2 *o = out + p0 * plane + (int64_t)y * W + x;
        const float xf = (float)(x + 1);
        float pf = (float)(p0 + 1);
        for (int64_t p = p0; p < p1; ++p, o += plane, pf += 1.f) __stcs(o, make_float2(pf, xf));
    }
}

cudaError_t launch_store_pattern(float2 *out, int64_t nplanes, int H, int W, int ctas, cudaStream_t st)
{
    k_store_pattern<<<ctas, 512, 0, st>>>(out, nplanes, H, W);
    return cudaGetLastError();
}

}  // namespace gb
