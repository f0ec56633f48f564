// Register-blocked 1-D Gaussian passes shared by the FP32 bank and SDFT kernels.
//
// Both passes are the real 1-D Gaussian smoothing S * g of the paper's decomposition
// (Eq. 5-6 along rows, Eq. 7-9 along columns): a thread produces 8 consecutive outputs,
// walks the taps in chunks of 8 (taps padded with zeros to a multiple of 8) and keeps a
// 16-sample window in registers, so every shared-memory load feeds 8 FMAs per signal.
#pragma once

#include <cuda_runtime.h>

namespace gb {

__device__ __forceinline__ float4 fma4(float4 w, float t, float4 a)
{
    return make_float4(fmaf(w.x, t, a.x), fmaf(w.y, t, a.y), fmaf(w.z, t, a.z), fmaf(w.w, t, a.w));
}
__device__ __forceinline__ float2 fma2(float2 w, float t, float2 a)
{
    return make_float2(fmaf(w.x, t, a.x), fmaf(w.y, t, a.y));
}
__device__ __forceinline__ float4 fmav(float4 w, float t, float4 a) { return fma4(w, t, a); }
__device__ __forceinline__ float2 fmav(float2 w, float t, float2 a) { return fma2(w, t, a); }

template <typename V> __device__ __forceinline__ V zero_v();
template <> __device__ __forceinline__ float4 zero_v<float4>() { return make_float4(0.f, 0.f, 0.f, 0.f); }
template <> __device__ __forceinline__ float2 zero_v<float2>() { return make_float2(0.f, 0.f); }

// Row pass: out[j] = sum_t src[j + t] * taps[t], j < 8, for two interleaved signals
// (f_c, f_s of Eq. 5).  src: 8 + 8 * nchunks readable float2; taps4: 2 * nchunks float4.
__device__ __forceinline__ void row_conv8(const float2 *__restrict__ src,
                                          const float4 *__restrict__ taps4, int nchunks,
                                          float2 (&acc)[8])
{
    float2 w[16];
#pragma unroll
    for (int i = 0; i < 8; ++i) w[i] = src[i];
#pragma unroll 2
    for (int c = 0; c < nchunks; ++c) {
#pragma unroll
        for (int i = 0; i < 8; ++i) w[8 + i] = src[8 * (c + 1) + i];
        const float4 t0 = taps4[2 * c], t1 = taps4[2 * c + 1];
        const float t[8] = {t0.x, t0.y, t0.z, t0.w, t1.x, t1.y, t1.z, t1.w};
#pragma unroll
        for (int d = 0; d < 8; ++d)
#pragma unroll
            for (int j = 0; j < 8; ++j) acc[j] = fma2(w[j + d], t[d], acc[j]);
#pragma unroll
        for (int i = 0; i < 8; ++i) w[i] = w[8 + i];
    }
}

// Column pass over a ring of rows: out[j] = sum_t ring[slot(j + t)][x] * taps[t], j < 8.
// V = float4 (four signals of an orientation pair) or float2 (one orientation).
// slot0 and RS are multiples of 8, so an 8-row chunk never wraps.
template <typename V>
__device__ __forceinline__ void col_conv8(const V *__restrict__ ring, int stride, int RS,
                                          int slot0, const float4 *__restrict__ taps4,
                                          int nchunks, V (&acc)[8])
{
    V w[16];
    int s = slot0;
#pragma unroll
    for (int i = 0; i < 8; ++i) w[i] = ring[(s + i) * stride];
#pragma unroll 2
    for (int c = 0; c < nchunks; ++c) {
        s += 8;
        if (s >= RS) s -= RS;
#pragma unroll
        for (int i = 0; i < 8; ++i) w[8 + i] = ring[(s + i) * stride];
        const float4 t0 = taps4[2 * c], t1 = taps4[2 * c + 1];
        const float t[8] = {t0.x, t0.y, t0.z, t0.w, t1.x, t1.y, t1.z, t1.w};
#pragma unroll
        for (int d = 0; d < 8; ++d)
#pragma unroll
            for (int j = 0; j < 8; ++j) acc[j] = fmav(w[j + d], t[d], acc[j]);
#pragma unroll
        for (int i = 0; i < 8; ++i) w[i] = w[8 + i];
    }
}

__host__ __device__ constexpr int round_up(int a, int b) { return (a + b - 1) / b * b; }

// Staging row width: at least need float2, and = 1 (mod 16) so that the 8 rows x 2 column
// groups of a half-warp fall on distinct bank pairs.
__host__ __device__ constexpr int stage_width(int need) { return round_up(need - 1, 16) + 1; }

}  // namespace gb
