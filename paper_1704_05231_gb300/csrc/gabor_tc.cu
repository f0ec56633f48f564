// Tensor-core Gabor filter bank (K6): Algorithm 1 of arXiv 1704.05231 with both 1-D Gaussian
// passes run as dense contractions on tcgen05 tensor cores (FP16 or BF16 operands, FP32
// accumulation in TMEM), the demodulation / remodulation and the orientation reuse in FP32.
//
// The 1-D Gaussian smoothing of a block of signals is a product with a banded Toeplitz
// matrix G[out][in] = S(in - out - offset), shared by every signal of a frequency, so each
// pass is a GEMM with a constant B operand:
//
//   row kernel     A[(r, c|s)][k] = f(y0 + r, x0 - R + k) (cos, sin)(w^c (x0 - R + k))  (Eq. 5)
//                  D[(r, c|s)][x] = sum_k A B_row[x][k]          -> S * f_c, S * f_s   (Eq. 5-6)
//                  epilogue: J = remodulation (Eq. 5-6), then the column signals of Eq. 10
//                  f_cr + f_si, f_sr - f_ci (theta) and f_cr - f_si, f_sr + f_ci (pi - theta,
//                  Eq. 15-16; J_{pi-theta} = J*_theta costs nothing), written transposed
//                  (image rows contiguous) to an FP16/BF16 intermediate that stays in L2.
//   column kernel  A[(signal, x)][l] = signal(x, y0 - R8 + l)
//                  D[(signal, x)][y] = sum_l A B_col[y][l]        -> P, Q, P', Q'         (Eq. 9)
//                  epilogue: F = remodulation by (cos, sin)(w^s y) (Eq. 7-8, 15-16), stored
//                  as complex64 with coalesced rows.
//
// Both kernels stage operands in the 128-byte-swizzled K-major layout, issue tcgen05.mma
// from one thread, wait on an mbarrier with a bounded wait, and read D with tcgen05.ld.
#include <algorithm>
#include <type_traits>

#include <cuda_fp16.h>
#include <cuda_bf16.h>

#include "internal.h"
#include "conv_fp32.cuh"
#include "tc_common.cuh"

namespace gb {

namespace {

template <typename T> __device__ __forceinline__ uint16_t tbits(float v);
template <> __device__ __forceinline__ uint16_t tbits<__half>(float v) { return __half_as_ushort(__float2half_rn(v)); }
template <> __device__ __forceinline__ uint16_t tbits<__nv_bfloat16>(float v)
{
    return __bfloat16_as_ushort(__float2bfloat16_rn(v));
}
template <typename T> __device__ __forceinline__ float tfloat(uint16_t b);
template <> __device__ __forceinline__ float tfloat<__half>(uint16_t b) { return __half2float(__ushort_as_half(b)); }
template <> __device__ __forceinline__ float tfloat<__nv_bfloat16>(uint16_t b)
{
    return __bfloat162float(__ushort_as_bfloat16(b));
}

constexpr int kTcTile = 64;   // rows per row-kernel tile; output rows per column-kernel tile

__device__ __forceinline__ void load_b(unsigned char *dst, const uint16_t *src, int bytes, int tid, int nthreads)
{
    const uint4 *s = reinterpret_cast<const uint4 *>(src);
    uint4 *d = reinterpret_cast<uint4 *>(dst);
    for (int i = tid; i < bytes / 16; i += nthreads) d[i] = s[i];
}

__device__ __forceinline__ void fail_status(int *status, volatile int *flag, int code)
{
    *flag = 1;
    atomicExch(status, code);
}

}  // namespace

// ------------------------------------------------------------------------------ row pass
// grid (ceil(W / 64), ceil(H / 64), units), 128 threads.
template <typename T>
__global__ void __launch_bounds__(128) k_gabor_tc_rows(const TcBankArgs a)
{
    extern __shared__ unsigned char smem_dyn[];
    unsigned char *sm = reinterpret_cast<unsigned char *>(((uintptr_t)smem_dyn + 1023) & ~(uintptr_t)1023);
    const TcUnitDev u = a.units[blockIdx.z];
    const TcFreqDev f = a.freqs[u.s];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int x0 = blockIdx.x * kTcTile, y0 = blockIdx.y * kTcTile;
    const int R = f.R, K = f.Krow;
    const int ncols = kTcTile + 2 * R;            // input columns x0 - R .. x0 + 63 + R
    const int PW = round_up(ncols, 4);

    unsigned char *sB = sm;                                       // 64 x K
    unsigned char *sA = sB + (size_t)kTcTile * K * 2;             // 128 x K (later: signal staging)
    float *patch = reinterpret_cast<float *>(sA + (size_t)128 * K * 2);     // 64 x PW
    float2 *ph = reinterpret_cast<float2 *>(patch + (size_t)kTcTile * PW);  // PW phases
    uint64_t *bar = reinterpret_cast<uint64_t *>(ph + PW + 2);
    uint32_t *tmem_s = reinterpret_cast<uint32_t *>(bar + 1);
    volatile int *flag = reinterpret_cast<volatile int *>(tmem_s + 1);
    float *wmax = reinterpret_cast<float *>(tmem_s + 2);          // [4]

    load_b(sB, f.Brow, kTcTile * K * 2, tid, 128);
    float m = 0.f;
    for (int r = warp; r < kTcTile; r += 4) {
        const int y = y0 + r;
        const bool yin = y < a.H;
        for (int c = lane; c < PW; c += 32) {
            const int gx = x0 - R + c;
            float v = 0.f;
            if (yin && c < ncols && gx >= 0 && gx < a.W) v = __ldg(a.img + (int64_t)y * a.pitch + gx);
            patch[r * PW + c] = v;
            m = fmaxf(m, fabsf(v));
        }
    }
    for (int c = tid; c < PW; c += 128) {
        const int gx = x0 - R + c;
        ph[c] = (c < ncols && gx >= 0 && gx < a.W) ? u.phx[gx] : make_float2(0.f, 0.f);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (lane == 0) wmax[warp] = m;
    if (tid == 0) {
        mbar_init(bar, 1);
        *flag = 0;
        mbar_fence_init();
    }
    if (warp == 0) {
        tmem_alloc(tmem_s, 64);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_s;
    const float mx = fmaxf(fmaxf(wmax[0], wmax[1]), fmaxf(wmax[2], wmax[3]));
    int e = 0;
    if (mx > 0.f) frexpf(mx, &e);
    const float sc = ldexpf(1.f, -e);

    // A[2r + sig][k] = f * (cos | sin) * 2^-e, K-major SW128, 8 k per 16-byte chunk.
    const int nchunk = 128 * (K / 8);
    for (int ci = tid; ci < nchunk; ci += 128) {
        const int row = ci & 127, kc = ci >> 7;
        const int r = row >> 1, sg = row & 1;
        uint32_t w[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int k0 = 8 * kc + 2 * q;
            float v0 = 0.f, v1 = 0.f;
            if (k0 < PW) {
                const float2 p0 = ph[k0];
                v0 = patch[r * PW + k0] * (sg ? p0.y : p0.x) * sc;
            }
            if (k0 + 1 < PW) {
                const float2 p1 = ph[k0 + 1];
                v1 = patch[r * PW + k0 + 1] * (sg ? p1.y : p1.x) * sc;
            }
            w[q] = (uint32_t)tbits<T>(v0) | ((uint32_t)tbits<T>(v1) << 16);
        }
        *reinterpret_cast<uint4 *>(sA + sw128_offset(128, row, 8 * kc)) = make_uint4(w[0], w[1], w[2], w[3]);
    }
    fence_proxy_async_smem();
    __syncthreads();
    if (tid == 0) {
        tc_fence_after();
        const uint32_t idesc = idesc_f16(std::is_same<T, __nv_bfloat16>::value ? 1 : 0, 128, kTcTile);
        const uint32_t a0 = smem_u32(sA), b0 = smem_u32(sB);
        for (int kb = 0; kb < K / 64; ++kb)
#pragma unroll
            for (int kk = 0; kk < 4; ++kk)
                tc_mma_f16(tmem, smem_desc_sw128(a0 + kb * 128 * 128) + 2 * kk,
                           smem_desc_sw128(b0 + kb * kTcTile * 128) + 2 * kk, idesc, (kb | kk) != 0);
        tc_commit(bar);
    }
    const bool done = mbar_wait(bar, 0, flag);
    if (!done && lane == 0) fail_status(a.status, flag, 11);
    tc_fence_after();

    // Epilogue: lane = A row 2r + sig (pairs of lanes hold S*f_c and S*f_s of one row r).
    uint16_t *stage = reinterpret_cast<uint16_t *>(sA);   // [4 signals][64 x][64 r]
    const int row = 32 * warp + lane;
    const int r = row >> 1, sg = row & 1;
    const int y = y0 + r;
    const bool yin = y < a.H;
    const float2 cy = yin ? u.phy[y] : make_float2(0.f, 0.f);
    const float unscale = ldexpf(f.unscale_row, e);
    const bool paired = u.plane_b >= 0;
    __syncthreads();   // A fully consumed by the MMAs before it is reused as staging
    for (int c0 = 0; c0 < kTcTile; c0 += 16) {
        float v[16];
        tmem_ld16(tmem + ((uint32_t)(32 * warp) << 16) + c0, v);
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            const float mine = v[j] * unscale;
            const float other = __shfl_xor_sync(0xffffffffu, mine, 1);
            const float A = sg ? other : mine, B = sg ? mine : other;
            const int x = c0 + j;
            const float2 px = ph[R + x];
            // Eq. 5-6: Re J = cos A + sin B, Im J = sin A - cos B
            const float jr = fmaf(px.x, A, px.y * B), ji = fmaf(px.y, A, -px.x * B);
            // Eq. 10
            const float fcr = jr * cy.x, fsr = jr * cy.y, fci = ji * cy.x, fsi = ji * cy.y;
            float s0, s1;
            if (sg == 0) { s0 = fcr + fsi; s1 = fsr - fci; }     // theta:      P_in, Q_in
            else         { s0 = fcr - fsi; s1 = fsr + fci; }     // pi - theta: P'_in, Q'_in
            if (!yin) { s0 = 0.f; s1 = 0.f; }
            if (sg == 0 || paired) {
                stage[((2 * sg) * kTcTile + x) * kTcTile + r] = tbits<T>(s0);
                stage[((2 * sg + 1) * kTcTile + x) * kTcTile + r] = tbits<T>(s1);
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    // Coalesced copy of the staged signals: one 128-byte row (64 image rows) per (signal, x).
    const int nsig = paired ? 4 : 2;
    const int nrow = nsig * kTcTile;
    for (int ci = tid; ci < nrow * 8; ci += 128) {
        const int nr = ci >> 3, ch = ci & 7;
        const int sgi = nr / kTcTile, x = nr % kTcTile;
        if (x0 + x < a.W) {
            const uint4 val = *reinterpret_cast<const uint4 *>(stage + nr * kTcTile + ch * 8);
            uint16_t *dst = a.sig + u.sig_off + ((int64_t)sgi * a.W + x0 + x) * a.Hp + a.Lpad + y0 + ch * 8;
            *reinterpret_cast<uint4 *>(dst) = val;
        }
    }
    if (warp == 0) tmem_dealloc(tmem, 64);
}

// --------------------------------------------------------------------------- column pass
// grid (items), 128 threads.  Item: unit, x0, y0; paired units take 32 columns x 4 signals,
// unpaired units 64 columns x 2 signals (both 128 A rows).
template <typename T>
__global__ void __launch_bounds__(128) k_gabor_tc_cols(const TcBankArgs a, const int4 *__restrict__ items)
{
    extern __shared__ unsigned char smem_dyn[];
    unsigned char *sm = reinterpret_cast<unsigned char *>(((uintptr_t)smem_dyn + 1023) & ~(uintptr_t)1023);
    const int4 it = items[blockIdx.x];
    const TcUnitDev u = a.units[it.x];
    const TcFreqDev f = a.freqs[u.s];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int x0 = it.y, y0 = it.z;
    const bool paired = u.plane_b >= 0;
    const int xw = paired ? 32 : 64;              // columns of this item
    const int K = f.Kcol;

    unsigned char *sB = sm;                                   // 64 x K
    unsigned char *sA = sB + (size_t)kTcTile * K * 2;         // 128 x K
    float *xch = reinterpret_cast<float *>(sA + (size_t)128 * K * 2);   // [2][64 y][32 x] (paired) or [64 y][64 x]
    float2 *phy = reinterpret_cast<float2 *>(xch + 2 * kTcTile * 32);   // 64 phases
    uint64_t *bar = reinterpret_cast<uint64_t *>(phy + kTcTile);
    uint32_t *tmem_s = reinterpret_cast<uint32_t *>(bar + 1);
    volatile int *flag = reinterpret_cast<volatile int *>(tmem_s + 1);

    // A rows n = signal * xw + x: the signal's column x, image rows y0 - R8 + l, l < K.
    const int nchunk = 128 * (K / 8);
    const int64_t lbase = (int64_t)a.Lpad + y0 - f.R8;
    for (int ci = tid; ci < nchunk; ci += 128) {
        const int n = ci & 127, kc = ci >> 7;
        const int sgi = n / xw, x = n % xw;
        const bool ok = x0 + x < a.W;
        const uint16_t *src = a.sig + u.sig_off + ((int64_t)sgi * a.W + (ok ? x0 + x : 0)) * a.Hp + lbase + 8 * kc;
        const unsigned s = smem_u32(sA + sw128_offset(128, n, 8 * kc));
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(s), "l"(src), "r"(ok ? 16 : 0) : "memory");
    }
    asm volatile("cp.async.commit_group;\n" ::: "memory");
    load_b(sB, f.Bcol, kTcTile * K * 2, tid, 128);
    for (int i = tid; i < kTcTile; i += 128) phy[i] = (y0 + i < a.H) ? u.phy[y0 + i] : make_float2(0.f, 0.f);
    if (tid == 0) {
        mbar_init(bar, 1);
        *flag = 0;
        mbar_fence_init();
    }
    if (warp == 0) {
        tmem_alloc(tmem_s, 64);
        tmem_relinquish();
    }
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");
    fence_proxy_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_s;
    if (tid == 0) {
        const uint32_t idesc = idesc_f16(std::is_same<T, __nv_bfloat16>::value ? 1 : 0, 128, kTcTile);
        const uint32_t a0 = smem_u32(sA), b0 = smem_u32(sB);
        for (int kb = 0; kb < K / 64; ++kb)
#pragma unroll
            for (int kk = 0; kk < 4; ++kk)
                tc_mma_f16(tmem, smem_desc_sw128(a0 + kb * 128 * 128) + 2 * kk,
                           smem_desc_sw128(b0 + kb * kTcTile * 128) + 2 * kk, idesc, (kb | kk) != 0);
        tc_commit(bar);
    }
    const bool done = mbar_wait(bar, 0, flag);
    if (!done && lane == 0) fail_status(a.status, flag, 12);
    tc_fence_after();

    // D[n][y]: warp w holds signal rows 32w .. 32w+31.
    //   paired:   warp 0 P, 1 Q (theta), 2 P', 3 Q' (pi - theta), x = lane
    //   unpaired: warps 0-1 P (x = 32 (w&1) + lane), warps 2-3 Q
    const float unscale = f.unscale_col;
    const bool is_q = paired ? (warp & 1) : (warp >= 2);
    const int slot = paired ? (warp >> 1) : (warp & 1);     // which exchange half
    if (is_q) {
        for (int c0 = 0; c0 < kTcTile; c0 += 16) {
            float v[16];
            tmem_ld16(tmem + ((uint32_t)(32 * warp) << 16) + c0, v);
#pragma unroll
            for (int j = 0; j < 16; ++j) xch[(slot * kTcTile + c0 + j) * 32 + lane] = v[j] * unscale;
        }
    }
    tc_fence_before();
    __syncthreads();
    if (!is_q) {
        const int x = x0 + (paired ? lane : 32 * slot + lane);
        const int plane = paired ? (slot == 0 ? u.plane_a : u.plane_b) : u.plane_a;
        float2 *o = a.out + (int64_t)plane * a.plane + x;
        for (int c0 = 0; c0 < kTcTile; c0 += 16) {
            float v[16];
            tmem_ld16(tmem + ((uint32_t)(32 * warp) << 16) + c0, v);
            if (x < a.W) {
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    const int yy = c0 + j;
                    if (y0 + yy < a.H) {
                        const float P = v[j] * unscale;
                        const float Q = xch[(slot * kTcTile + yy) * 32 + lane];
                        const float2 t = phy[yy];
                        // Eq. 7-8 (theta) and Eq. 15-16 (pi - theta)
                        __stcs(o + (int64_t)(y0 + yy) * a.W, make_float2(fmaf(t.x, P, t.y * Q), fmaf(t.y, P, -t.x * Q)));
                    }
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0) tmem_dealloc(tmem, 64);
}

// ------------------------------------------------------------------------ Toeplitz B (FP64)
// B[j][k] = S(k - j - off) * 2^sB for |k - j - off| <= R, rows j < 64, K-major SW128.
__global__ void k_build_toeplitz(uint16_t *__restrict__ B, int K, int off, int R, double sigma, int sB, int bf16)
{
    const int n = kTcTile * K;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int j = i / K, k = i % K;
        const int d = k - j - off;
        double v = 0.0;
        if (d >= -R && d <= R) v = ldexp(exp(-(double)d * d / (2.0 * sigma * sigma)) / (2.5066282746310002 * sigma), sB);
        const float fv = (float)v;
        B[sw128_offset(kTcTile, j, k) / 2] = bf16 ? __bfloat16_as_ushort(__float2bfloat16_rn(fv)) : __half_as_ushort(__float2half_rn(fv));
    }
}

TcGeometry gabor_tc_geometry(int R)
{
    TcGeometry g;
    g.R = R;
    g.R8 = round_up(R, 8);
    g.Krow = round_up(kTcTile + 2 * R, 64);
    g.Kcol = round_up(kTcTile + g.R8 + R, 64);
    const int PW = round_up(kTcTile + 2 * R, 4);
    g.smem_rows = 1024 + (size_t)kTcTile * g.Krow * 2 + (size_t)128 * g.Krow * 2 + (size_t)kTcTile * PW * 4 +
                  (size_t)(PW + 2) * 8 + 64;
    g.smem_cols = 1024 + (size_t)kTcTile * g.Kcol * 2 + (size_t)128 * g.Kcol * 2 + (size_t)2 * kTcTile * 32 * 4 +
                  (size_t)kTcTile * 8 + 64;
    return g;
}

bool gabor_tc_supported(int R)
{
    const TcGeometry g = gabor_tc_geometry(R);
    return g.smem_rows <= (size_t)kSmemLimit && g.smem_cols <= (size_t)kSmemLimit && g.Kcol <= 512;
}

cudaError_t build_gabor_tc_b(uint16_t *Brow, uint16_t *Bcol, int R, double sigma, int bf16, float *unscale,
                             cudaStream_t st)
{
    const TcGeometry g = gabor_tc_geometry(R);
    // max S = S(0) = 1 / (sqrt(2 pi) sigma): scale into [0.5, 1)
    int e = 0;
    frexp(1.0 / (2.5066282746310002 * sigma), &e);
    const int sB = -e;
    *unscale = (float)ldexp(1.0, -sB);
    k_build_toeplitz<<<(kTcTile * g.Krow + 255) / 256, 256, 0, st>>>(Brow, g.Krow, R, R, sigma, sB, bf16);
    cudaError_t err = cudaGetLastError();
    if (err != cudaSuccess) return err;
    k_build_toeplitz<<<(kTcTile * g.Kcol + 255) / 256, 256, 0, st>>>(Bcol, g.Kcol, g.R8, R, sigma, sB, bf16);
    return cudaGetLastError();
}

cudaError_t gabor_tc_prepare()
{
    cudaError_t e = cudaSuccess;
    const void *fns[4] = {(const void *)k_gabor_tc_rows<__half>, (const void *)k_gabor_tc_rows<__nv_bfloat16>,
                          (const void *)k_gabor_tc_cols<__half>, (const void *)k_gabor_tc_cols<__nv_bfloat16>};
    for (const void *fn : fns)
        if (e == cudaSuccess) e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemLimit);
    return e;
}

cudaError_t launch_gabor_tc(const TcBankArgs &a, int nunits, size_t smem_rows, size_t smem_cols, const int4 *items,
                            int nitems, int bf16, cudaStream_t st)
{
    const dim3 grid_r((a.W + kTcTile - 1) / kTcTile, (a.H + kTcTile - 1) / kTcTile, nunits);
    if (bf16)
        k_gabor_tc_rows<__nv_bfloat16><<<grid_r, 128, smem_rows, st>>>(a);
    else
        k_gabor_tc_rows<__half><<<grid_r, 128, smem_rows, st>>>(a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || nitems == 0) return e;
    if (bf16)
        k_gabor_tc_cols<__nv_bfloat16><<<nitems, 128, smem_cols, st>>>(a, items);
    else
        k_gabor_tc_cols<__half><<<nitems, 128, smem_cols, st>>>(a, items);
    return cudaGetLastError();
}

}  // namespace gb
