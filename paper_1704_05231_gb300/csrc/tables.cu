// K0: FP64 table builder.  The only double-precision arithmetic on the GPU: modulation
// phases of Eq. 5-10 (cos / sin of omega cos(theta) x and omega sin(theta) y), the sampled
// Gaussian S_sigma(d) of Sec. II, and the SDFT twiddles of Eq. 18.  Results are stored as
// FP32 for the FP32 kernels.
//
// Phase reduction: the argument a = omega cos(theta) x is formed as r = (omega cos(theta) /
// pi) * x and reduced exactly modulo 2 (fmod is exact), then sincospi(r) is evaluated.  The
// reduction is exact whenever omega cos(theta) / pi is a dyadic rational (theta = 0 or pi/2
// with omega = pi / 2^k); otherwise the only error is the rounding of one product in FP64.
// SDFT twiddles use the integer index j = (u m) mod M and sincospi(2 j / M).
#include "internal.h"

namespace gb {

__global__ void k_build_gabor_tables(const double *__restrict__ unit_w, int nunits, int Wcap,
                                     int Hcap, int mg, float2 *__restrict__ phx, float2 *__restrict__ phy)
{
    const int64_t wx = (int64_t)Wcap + 2 * mg, wy = (int64_t)Hcap + 2 * mg;
    const int64_t per = wx + wy;
    const int64_t n = per * nunits;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int u = (int)(i / per);
        const int64_t p = i % per;
        const bool is_x = p < wx;
        const double c = is_x ? unit_w[2 * u] : unit_w[2 * u + 1];
        const double pos = (double)((is_x ? p : p - wx) - mg);   // may be negative
        double r = fmod(c * pos, 2.0);
        double s, co;
        sincospi(r, &s, &co);
        const float2 v = make_float2((float)co, (float)s);
        if (is_x)
            phx[(int64_t)u * wx + p] = v;
        else
            phy[(int64_t)u * wy + (p - wx)] = v;
    }
}

// S(d) = exp(-d^2 / (2 sigma^2)) / (sqrt(2 pi) sigma) in FP64, rounded to FP32 (Sec. II).
__device__ __forceinline__ float gauss_tap(double d, double sg)
{
    return (float)(exp(-(d * d) / (2.0 * sg * sg)) / (2.5066282746310002 * sg));
}

// taps[s][t] = S_sigma_s(t - lo_s) for t < T_s, zero for T_s <= t < tpad_max.
__global__ void k_build_taps(const double *__restrict__ sigma, const int *__restrict__ lo,
                             const int *__restrict__ T, int nfreq, int tpad_max,
                             float *__restrict__ taps)
{
    const int n = nfreq * tpad_max;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int s = i / tpad_max, t = i % tpad_max;
        taps[i] = t < T[s] ? gauss_tap((double)(t - lo[s]), sigma[s]) : 0.f;
    }
}

__global__ void k_build_twiddles(int M, float2 *__restrict__ tw)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j < M) {
        double s, c;
        sincospi(2.0 * (double)j / (double)M, &s, &c);
        tw[j] = make_float2((float)c, (float)s);
    }
}

// Every table of the FP32 SDFT from parameters passed by value (no device inputs): taps of
// both window axes, taps[a][t] = S_sigma(t - M_a / 2) for t < M_a and 0 up to tap_stride, and
// the twiddles tw[a][j] = (cos, sin)(2 pi j / M_a) for j < M_a and (1, 0) up to tw_stride
// (a = 0: x, M_0 = Mx; a = 1: y, M_1 = My).  The same values as k_build_taps and
// k_build_twiddles, entry for entry.
__global__ void k_build_sdft_tables(double sigma, int Mx, int My, int tap_stride, int tw_stride,
                                    float *__restrict__ taps, float2 *__restrict__ tw)
{
    const int ntap = 2 * tap_stride, n = ntap + 2 * tw_stride;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        if (i < ntap) {
            const int ax = i / tap_stride, t = i % tap_stride;
            const int M = ax ? My : Mx;
            taps[i] = t < M ? gauss_tap((double)(t - M / 2), sigma) : 0.f;
        } else {
            const int k = i - ntap, ax = k / tw_stride, j = k % tw_stride;
            const int M = ax ? My : Mx;
            double sn = 0.0, c = 1.0;
            if (j < M) sincospi(2.0 * (double)j / (double)M, &sn, &c);
            tw[k] = make_float2((float)c, (float)sn);
        }
    }
}

cudaError_t launch_build_sdft_tables(double sigma, int Mx, int My, int tap_stride, int tw_stride, float *taps,
                                     float2 *tw, cudaStream_t st)
{
    const int n = 2 * (tap_stride + tw_stride);
    k_build_sdft_tables<<<(n + 255) / 256, 256, 0, st>>>(sigma, Mx, My, tap_stride, tw_stride, taps, tw);
    return cudaGetLastError();
}

cudaError_t launch_build_gabor_tables(const double *d_unit_w, int nunits, int Wcap, int Hcap, int mg,
                                      float2 *phx, float2 *phy, cudaStream_t st)
{
    if (nunits == 0) return cudaSuccess;
    const int64_t n = ((int64_t)Wcap + Hcap + 4 * mg) * nunits;
    const int blocks = (int)std::min<int64_t>((n + 255) / 256, 4096);
    k_build_gabor_tables<<<blocks, 256, 0, st>>>(d_unit_w, nunits, Wcap, Hcap, mg, phx, phy);
    return cudaGetLastError();
}

cudaError_t launch_build_taps(const double *d_sigma, const int *d_lo, const int *d_T, int nfreq,
                              int tpad_max, float *taps, cudaStream_t st)
{
    if (nfreq == 0) return cudaSuccess;
    const int n = nfreq * tpad_max;
    k_build_taps<<<(n + 255) / 256, 256, 0, st>>>(d_sigma, d_lo, d_T, nfreq, tpad_max, taps);
    return cudaGetLastError();
}

cudaError_t launch_build_twiddles(int M, float2 *tw, cudaStream_t st)
{
    k_build_twiddles<<<(M + 63) / 64, 64, 0, st>>>(M, tw);
    return cudaGetLastError();
}

}  // namespace gb
