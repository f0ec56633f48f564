// Tensor-core Gabor filter bank (K6): Algorithm 1 of arXiv 1704.05231 with both 1-D Gaussian
// passes run as dense contractions on tcgen05 tensor cores (FP16 operands, FP32 accumulation
// in TMEM); demodulation, remodulation and the orientation reuse stay in FP32.
//
// The 1-D Gaussian smoothing of a block of signals is a product with a banded Toeplitz matrix
// G[out][in] = S(in - out - offset), shared by every signal of a frequency:
//
//   row kernel     D[x][(r, c|s)] = sum_k T[x][k] Dm[(r, c|s)][k],  T[x][k] = S(k - x - R),
//                  Dm = f(y0 + r, x0 - R + k) (cos, sin)(w^c (x0 - R + k))          (Eq. 5)
//                  -> S * f_c, S * f_s for 128 columns x 64 rows of one unit.   Epilogue
//                  (thread = one image column): J = remodulation (Eq. 5-6), the column
//                  signals of Eq. 10, f_cr + f_si, f_sr - f_ci (theta) and f_cr - f_si,
//                  f_sr + f_ci (pi - theta, Eq. 15-16: J_{pi-theta} = J*_theta costs nothing),
//                  written as FP16 with image rows contiguous (16-byte stores) to an
//                  intermediate that stays in L2.
//   column kernel  D[(signal, x)][y] = sum_l Sig[(signal, x)][l] G[y][l],  G[y][l] = S(l - y - R8)
//                  -> P, Q, P', Q' (Eq. 9).  Epilogue: F = remodulation by (cos, sin)(w^s y)
//                  (Eq. 7-8, 15-16), complex64 stores with coalesced rows.
//
// Both kernels are persistent (one CTA per SM) and warp-specialised: warps 4-7 stage operands
// in the 128-byte-swizzled K-major layout and thread 128 issues tcgen05.mma into one of two TMEM
// buffers; warps 0-3 read the accumulators with tcgen05.ld.  Every mbarrier wait is bounded.
#include <algorithm>
#include <type_traits>

#include <cuda_fp16.h>

#include "internal.h"
#include "conv_fp32.cuh"
#include "tc_common.cuh"

namespace gb {

namespace {

constexpr int kRowTileX = 128;   // row kernel: image columns per tile (MMA M)
constexpr int kRowTileYMax = 64; // row kernel: image rows per tile (64, or 32 for large radii; MMA N = 2 x rows)
constexpr int kColTileY = 64;    // column kernel: output rows per tile (MMA N)

__device__ __forceinline__ uint16_t h16(float v) { return __half_as_ushort(__float2half_rn(v)); }

__device__ __forceinline__ void fail_status(int *status, volatile int *flag, int code)
{
    *flag = 1;
    atomicExch(status, code);
}

struct RowSmem {
    uint32_t t_off, dm_off, patch_off, ph_off, bar_off, misc_off, total;
};

__host__ __device__ inline RowSmem row_smem(int K, int PW, int TY)
{
    RowSmem L;
    L.t_off = 0;
    L.dm_off = L.t_off + (uint32_t)kRowTileX * K * 2;
    L.patch_off = L.dm_off + (uint32_t)(2 * TY) * K * 2;
    L.ph_off = L.patch_off + (uint32_t)TY * (round_up(PW, 8) + 4) * 4;
    L.bar_off = (L.ph_off + (uint32_t)PW * 8 + 15) & ~15u;
    L.misc_off = L.bar_off + 8 * 8;
    L.total = L.misc_off + 64;
    return L;
}

struct ColSmem {
    uint32_t g_off, a_off, xch_off, bar_off, misc_off, total;
};

__host__ __device__ inline ColSmem col_smem(int K)
{
    ColSmem L;
    L.g_off = 0;
    L.a_off = L.g_off + (uint32_t)kColTileY * K * 2;
    L.xch_off = L.a_off + 2u * 128 * K * 2;
    L.bar_off = L.xch_off + 2u * kColTileY * 32 * 4;
    L.misc_off = L.bar_off + 8 * 8;
    L.total = L.misc_off + 64;
    return L;
}

}  // namespace

// ------------------------------------------------------------------------- work items
// Items are decoded from the image shape: per frequency (largest radius first), the row pass
// has row_cnt tiles (TY rows x 128 columns); the column pass has, per unit, col_ny tiles of
// 64 rows x 32 columns (paired units, listed first) or x 64 columns (unpaired units).
struct RowItem {
    int s, y0, x0;
};
struct ColItem {
    int unit, x0, y0;
};
__device__ __forceinline__ RowItem row_item(const TcBankArgs &a, int it)
{
    const int g = it / a.row_cnt, local = it - g * a.row_cnt;
    return RowItem{__ldg(a.forder + g), (local / a.row_nx) * a.row_ty, (local % a.row_nx) * kRowTileX};
}
__device__ __forceinline__ ColItem col_item(const TcBankArgs &a, int it)
{
    const int g = it / a.col_cnt;
    int local = it - g * a.col_cnt;
    const int u0 = a.freqs[__ldg(a.forder + g)].u0;
    const int paired_items = a.np_f * a.col_ny * a.col_nx32;
    const bool paired = local < paired_items;
    if (!paired) local -= paired_items;
    const int nx = paired ? a.col_nx32 : a.col_nx64;
    const int per = a.col_ny * nx, q = local / per, r = local - q * per;
    return ColItem{u0 + (paired ? 0 : a.np_f) + q, (r % nx) * (paired ? 32 : 64), (r / nx) * kColTileY};
}

// ------------------------------------------------------------------------------ row pass
// Items: (frequency s, tile y, tile x), sorted by frequency; each item runs every unit of s.
// The input scale 2^-e (|f| 2^-e < 1, FP16 range) comes from k_absmax for the whole image.
__global__ void __launch_bounds__(384, 1) k_gabor_tc_rows(const __grid_constant__ TcBankArgs a)
{
    const int nitems = a.nf * a.row_cnt;
    extern __shared__ unsigned char smem_dyn[];
    unsigned char *sm = reinterpret_cast<unsigned char *>(((uintptr_t)smem_dyn + 1023) & ~(uintptr_t)1023);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int TY = a.row_ty;                 // image rows per tile
    const RowSmem L = row_smem(a.row_kmax, a.row_pwmax, TY);
    unsigned char *sT = sm + L.t_off;
    unsigned char *sDm = sm + L.dm_off;
    float *patch = reinterpret_cast<float *>(sm + L.patch_off);
    float2 *ph = reinterpret_cast<float2 *>(sm + L.ph_off);
    uint64_t *bars = reinterpret_cast<uint64_t *>(sm + L.bar_off);
    uint64_t *tmem_full = bars;        // [2] commit
    uint64_t *tmem_empty = bars + 2;   // [2] 4 epilogue warps
    uint64_t *dm_empty = bars + 4;     // [1] commit: the MMA reading Dm is done
    uint64_t *drain = bars + 5;
    uint32_t *tmem_s = reinterpret_cast<uint32_t *>(sm + L.misc_off);
    volatile int *abort_s = reinterpret_cast<volatile int *>(sm + L.misc_off + 4);

    if (tid == 0) {
        mbar_init(&tmem_full[0], 1);
        mbar_init(&tmem_full[1], 1);
        mbar_init(&tmem_empty[0], 4);
        mbar_init(&tmem_empty[1], 4);
        mbar_init(dm_empty, 1);
        mbar_init(drain, 1);
        *abort_s = 0;
        mbar_fence_init();
    }
    if (warp == 0) {
        tmem_alloc(tmem_s, 256);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_s;
    const uint32_t idesc = idesc_f16(0, kRowTileX, 2 * TY);
    int e = 0;
    {
        const float mx = __int_as_float(*a.absmax);
        if (mx > 0.f) frexpf(mx, &e);   // mx = m 2^e, m in [0.5, 1)
    }

    if (warp >= 4) {
        // -------------------------------------------------------------- producers
        constexpr int NP = 256;                 // producer threads (warps 4-11)
        const int ptid = tid - 128, pwarp = warp - 4;
        const float sc = ldexpf(1.f, -e);
        int cur_s = -1, job = 0;
        for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
            if (named_barrier_or(1, NP, *abort_s != 0)) break;
            const RowItem w = row_item(a, it);
            const int s = w.s, y0 = w.y0, x0 = w.x0;
            const TcFreqDev f = a.freqs[s];
            const int R = f.R, K = f.Krow;
            const int ncols = kRowTileX + 2 * R, PW = round_up(ncols, 4);
            const int PWs = round_up(PW, 8) + 4;     // row stride: 16-byte rows fall on distinct banks
            // The previous item's last MMA (which read Dm, and T) must be complete.
            bool failed = job > 0 && !mbar_wait(dm_empty, (job - 1) & 1, abort_s);
            if (named_barrier_or(1, NP, failed)) {
                if (ptid == 0) fail_status(a.status, abort_s, 21);
                break;
            }
            if (s != cur_s) {
                const uint4 *src = reinterpret_cast<const uint4 *>(f.Brow);
                uint4 *dst = reinterpret_cast<uint4 *>(sT);
                for (int i = ptid; i < kRowTileX * K * 2 / 16; i += NP) dst[i] = src[i];
                cur_s = s;
            }
            // patch rows y0 .. y0 + 63, columns x0 - R .. x0 + 127 + R (zero outside the image)
            for (int r = pwarp; r < TY; r += NP / 32) {
                const int y = y0 + r;
                const bool yin = y < a.H;
                const float *src = a.img + (int64_t)(yin ? y : 0) * a.pitch;
                for (int c = lane; c < PW; c += 32) {
                    const int gx = x0 - R + c;
                    const bool ok = yin && c < ncols && gx >= 0 && gx < a.W;
                    cp_async4(patch + r * PWs + c, ok ? (const void *)(src + gx) : (const void *)a.img, ok ? 4 : 0);
                }
            }
            cp_async_commit();
            cp_async_wait<0>();
            const int u0 = f.u0, nu = a.nu_f;
            bool stop = false;
            for (int q = 0; q < nu; ++q, ++job) {
                const TcUnitDev u = a.units[u0 + q];
                const int b = job & 1;
                // Dm is read by the previous job's MMA.
                failed = q > 0 && !mbar_wait(dm_empty, (job - 1) & 1, abort_s);
                if (named_barrier_or(1, NP, failed)) {
                    if (ptid == 0) fail_status(a.status, abort_s, 22);
                    stop = true;
                    break;
                }
                // demodulation phases times the input scale (Eq. 5)
                for (int c = ptid; c < PW; c += NP) {
                    const int gx = x0 - R + c;
                    const float2 v = (c < ncols && gx >= 0 && gx < a.W) ? u.phx[gx] : make_float2(0.f, 0.f);
                    ph[c] = make_float2(v.x * sc, v.y * sc);
                }
                named_barrier(1, NP);
                // Dm[n = 2r + sg][k]: a warp takes 32 rows n of one 8-k chunk (conflict-free
                // patch rows, broadcast phases, conflict-free swizzled stores).
                const int kch = K / 8;
#pragma unroll 2
                for (int ci = ptid; ci < 2 * TY * kch; ci += NP) {
                    const int n = ci % (2 * TY), kc = ci / (2 * TY);
                    const int r = n >> 1, sg = n & 1;
                    const int k0 = 8 * kc;
                    uint32_t wv[4];
                    if (k0 + 8 <= PW) {
                        const float4 p0 = *reinterpret_cast<const float4 *>(patch + r * PWs + k0);
                        const float4 p1 = *reinterpret_cast<const float4 *>(patch + r * PWs + k0 + 4);
                        const float pv[8] = {p0.x, p0.y, p0.z, p0.w, p1.x, p1.y, p1.z, p1.w};
#pragma unroll
                        for (int qq = 0; qq < 4; ++qq) {
                            const float2 h0 = ph[k0 + 2 * qq], h1 = ph[k0 + 2 * qq + 1];
                            const float v0 = pv[2 * qq] * (sg ? h0.y : h0.x);
                            const float v1 = pv[2 * qq + 1] * (sg ? h1.y : h1.x);
                            wv[qq] = (uint32_t)h16(v0) | ((uint32_t)h16(v1) << 16);
                        }
                    } else {
#pragma unroll
                        for (int qq = 0; qq < 4; ++qq) {
                            float vv[2];
#pragma unroll
                            for (int t2 = 0; t2 < 2; ++t2) {
                                const int k = k0 + 2 * qq + t2;
                                float v = 0.f;
                                if (k < PW) {
                                    const float2 h = ph[k];
                                    v = patch[r * PWs + k] * (sg ? h.y : h.x);
                                }
                                vv[t2] = v;
                            }
                            wv[qq] = (uint32_t)h16(vv[0]) | ((uint32_t)h16(vv[1]) << 16);
                        }
                    }
                    *reinterpret_cast<uint4 *>(sDm + sw128_offset(2 * TY, n, k0)) =
                        make_uint4(wv[0], wv[1], wv[2], wv[3]);
                }
                fence_proxy_async_smem();
                named_barrier(1, NP);
                if (ptid == 0) {
                    if (job >= 2 && !mbar_wait(&tmem_empty[b], ((job - 2) >> 1) & 1, abort_s)) {
                        fail_status(a.status, abort_s, 23);
                    } else {
                        tc_fence_after();
                        const uint32_t a0 = smem_u32(sT), b0 = smem_u32(sDm);
                        for (int kb = 0; kb < K / 64; ++kb)
#pragma unroll
                            for (int kk = 0; kk < 4; ++kk)
                                tc_mma_f16(tmem + 128u * b, smem_desc_sw128(a0 + kb * kRowTileX * 128) + 2 * kk,
                                           smem_desc_sw128(b0 + kb * (2 * TY) * 128) + 2 * kk, idesc,
                                           (kb | kk) != 0);
                        tc_commit(&tmem_full[b]);
                        tc_commit(dm_empty);
                    }
                }
            }
            if (stop) break;
        }
        if (ptid == 0) {
            tc_commit(drain);
            if (!mbar_wait(drain, 0, abort_s)) {
                volatile int dummy = 0;
                mbar_wait(drain, 0, &dummy);
            }
        }
    } else {
        // -------------------------------------------------------------- epilogue
        // Thread = image column x0 + x (TMEM lane x); accumulator columns 2r + {c, s}.
        const int x = 32 * warp + lane;
        const uint32_t lane_base = (uint32_t)(32 * warp) << 16;
        int job = 0;
        for (int it = blockIdx.x; it < nitems && !*abort_s; it += gridDim.x) {
            const RowItem w = row_item(a, it);
            const int y0 = w.y0;
            const TcFreqDev f = a.freqs[w.s];
            const float unscale = ldexpf(f.unscale_row, e);
            const int gx = w.x0 + x;
            const bool xin = gx < a.W;
            const int u0 = f.u0, nu = a.nu_f;
            bool ok = true;
            for (int q = 0; q < nu; ++q, ++job) {
                const TcUnitDev u = a.units[u0 + q];
                const int b = job & 1;
                // row phases of the tile, lane l holds rows l and l + 32 (broadcast by shuffle)
                const float2 py0 = (y0 + lane < a.H) ? __ldg(&u.phy[y0 + lane]) : make_float2(0.f, 0.f);
                const float2 py1 = (y0 + 32 + lane < a.H) ? __ldg(&u.phy[y0 + 32 + lane]) : make_float2(0.f, 0.f);
                const float2 px = xin ? __ldg(&u.phx[gx]) : make_float2(0.f, 0.f);
                if (!mbar_wait(&tmem_full[b], (job >> 1) & 1, abort_s)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const bool paired = u.plane_b >= 0;
                const int64_t sstride = (int64_t)a.W * a.Hp;   // between signals of the unit
                uint16_t *dst0 = a.sig + u.sig_idx * sstride + (int64_t)(xin ? gx : 0) * a.Hp + a.Lpad + y0;
#pragma unroll 1
                for (int c0 = 0; c0 < 2 * TY; c0 += 16) {
                    float v[16];
                    tmem_ld16(tmem + lane_base + 128u * b + c0, v);
                    const int r0 = c0 >> 1;
                    uint32_t pk[4][4];
#pragma unroll
                    for (int j = 0; j < 8; ++j) {
                        const int r = r0 + j;
                        const float2 pyr = r < 32 ? py0 : py1;
                        const float2 cy = make_float2(__shfl_sync(0xffffffffu, pyr.x, r & 31),
                                                      __shfl_sync(0xffffffffu, pyr.y, r & 31));
                        const float A = v[2 * j] * unscale, B = v[2 * j + 1] * unscale;
                        // Eq. 5-6: Re J = cos A + sin B, Im J = sin A - cos B
                        const float jr = fmaf(px.x, A, px.y * B), ji = fmaf(px.y, A, -px.x * B);
                        // Eq. 10
                        const float fcr = jr * cy.x, fsr = jr * cy.y, fci = ji * cy.x, fsi = ji * cy.y;
                        const uint32_t s0 = h16(fcr + fsi), s1 = h16(fsr - fci);
                        const uint32_t s2 = h16(fcr - fsi), s3 = h16(fsr + fci);
                        if ((j & 1) == 0) {
                            pk[0][j >> 1] = s0; pk[1][j >> 1] = s1; pk[2][j >> 1] = s2; pk[3][j >> 1] = s3;
                        } else {
                            pk[0][j >> 1] |= s0 << 16; pk[1][j >> 1] |= s1 << 16;
                            pk[2][j >> 1] |= s2 << 16; pk[3][j >> 1] |= s3 << 16;
                        }
                    }
                    if (xin) {
                        *reinterpret_cast<uint4 *>(dst0 + r0) = make_uint4(pk[0][0], pk[0][1], pk[0][2], pk[0][3]);
                        *reinterpret_cast<uint4 *>(dst0 + sstride + r0) = make_uint4(pk[1][0], pk[1][1], pk[1][2], pk[1][3]);
                        if (paired) {
                            *reinterpret_cast<uint4 *>(dst0 + 2 * sstride + r0) =
                                make_uint4(pk[2][0], pk[2][1], pk[2][2], pk[2][3]);
                            *reinterpret_cast<uint4 *>(dst0 + 3 * sstride + r0) =
                                make_uint4(pk[3][0], pk[3][1], pk[3][2], pk[3][3]);
                        }
                    }
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(&tmem_empty[b]);
            }
            if (!ok) {
                if (lane == 0) fail_status(a.status, abort_s, 24);
                break;
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0) tmem_dealloc(tmem, 256);
}

// --------------------------------------------------------------------------- column pass
// Items: (unit, x0, y0), sorted by frequency; paired units take 32 columns x 4 signals,
// unpaired ones 64 columns x 2 signals (always 128 A rows).  The producers keep one job of
// operand loads in flight ahead of the MMA.
__global__ void __launch_bounds__(256, 1) k_gabor_tc_cols(const __grid_constant__ TcBankArgs a)
{
    const int nitems = a.nf * a.col_cnt;
    extern __shared__ unsigned char smem_dyn[];
    unsigned char *sm = reinterpret_cast<unsigned char *>(((uintptr_t)smem_dyn + 1023) & ~(uintptr_t)1023);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const ColSmem L = col_smem(a.col_kmax);
    unsigned char *sG = sm + L.g_off;
    unsigned char *sA = sm + L.a_off;                 // [2] buffers of 128 x Kmax
    float *xch = reinterpret_cast<float *>(sm + L.xch_off);
    uint64_t *bars = reinterpret_cast<uint64_t *>(sm + L.bar_off);
    uint64_t *tmem_full = bars;        // [2]
    uint64_t *tmem_empty = bars + 2;   // [2] 4 epilogue warps
    uint64_t *a_empty = bars + 4;      // [2] commit
    uint64_t *drain = bars + 6;
    uint32_t *tmem_s = reinterpret_cast<uint32_t *>(sm + L.misc_off);
    volatile int *abort_s = reinterpret_cast<volatile int *>(sm + L.misc_off + 4);
    const uint32_t abuf = 128u * a.col_kmax * 2;

    if (tid == 0) {
        mbar_init(&tmem_full[0], 1);
        mbar_init(&tmem_full[1], 1);
        mbar_init(&tmem_empty[0], 4);
        mbar_init(&tmem_empty[1], 4);
        mbar_init(&a_empty[0], 1);
        mbar_init(&a_empty[1], 1);
        mbar_init(drain, 1);
        *abort_s = 0;
        mbar_fence_init();
    }
    if (warp == 0) {
        tmem_alloc(tmem_s, 128);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_s;
    const uint32_t idesc = idesc_f16(0, 128, kColTileY);
    const int njobs = nitems > (int)blockIdx.x ? (nitems - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;

    if (warp >= 4) {
        // -------------------------------------------------------------- producers
        const int ptid = tid - 128;
        auto item = [&](int j) { return col_item(a, blockIdx.x + j * gridDim.x); };
        auto load_g = [&](int s) {
            const TcFreqDev f = a.freqs[s];
            const uint4 *src = reinterpret_cast<const uint4 *>(f.Bcol);
            uint4 *dst = reinterpret_cast<uint4 *>(sG);
            for (int i = ptid; i < kColTileY * f.Kcol * 2 / 16; i += 128) dst[i] = src[i];
        };
        // cp.async of job j's A operand into buffer j & 1 (zero rows beyond the image).
        auto issue = [&](int j) {
            const ColItem w = item(j);
            const TcUnitDev u = a.units[w.unit];
            const TcFreqDev f = a.freqs[u.s];
            const int x0 = w.x0, y0 = w.y0, K = f.Kcol;
            const int xw = u.plane_b >= 0 ? 32 : 64;
            const int64_t lbase = (int64_t)a.Lpad + y0 - f.R8;
            unsigned char *dstA = sA + (j & 1) * abuf;
            const int kch = K / 8;
            for (int ci = ptid; ci < 128 * kch; ci += 128) {
                const int n = ci / kch, kc = ci - n * kch;
                const int sgi = n / xw, x = n - sgi * xw;
                const bool ok = x0 + x < a.W;
                const uint16_t *src =
                    a.sig + ((u.sig_idx + sgi) * a.W + (ok ? x0 + x : 0)) * a.Hp + lbase + 8 * kc;
                const unsigned sdst = smem_u32(dstA + sw128_offset(128, n, 8 * kc));
                asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(sdst), "l"(src), "r"(ok ? 16 : 0)
                             : "memory");
            }
            cp_async_commit();
        };
        auto freq_of = [&](int j) { return a.units[item(j).unit].s; };
        if (njobs > 0) {
            load_g(freq_of(0));
            issue(0);
        }
        for (int j = 0; j < njobs; ++j) {
            if (named_barrier_or(1, 128, *abort_s != 0)) break;
            const int sj = freq_of(j);
            const bool has_next = j + 1 < njobs;
            const bool same = has_next && freq_of(j + 1) == sj;
            bool failed = false;
            if (same) {
                // buffer (j+1)&1 was read by job j-1's MMA
                failed = j >= 1 && !mbar_wait(&a_empty[(j + 1) & 1], ((j - 1) >> 1) & 1, abort_s);
                if (named_barrier_or(1, 128, failed)) {
                    if (ptid == 0) fail_status(a.status, abort_s, 31);
                    break;
                }
                issue(j + 1);
                cp_async_wait<1>();
            } else {
                cp_async_wait<0>();
            }
            fence_proxy_async_smem();
            named_barrier(1, 128);
            if (ptid == 0) {
                const int b = j & 1;
                const TcFreqDev f = a.freqs[sj];
                if (j >= 2 && !mbar_wait(&tmem_empty[b], ((j - 2) >> 1) & 1, abort_s)) {
                    fail_status(a.status, abort_s, 32);
                } else {
                    tc_fence_after();
                    const uint32_t a0 = smem_u32(sA + b * abuf), g0 = smem_u32(sG);
                    for (int kb = 0; kb < f.Kcol / 64; ++kb)
#pragma unroll
                        for (int kk = 0; kk < 4; ++kk)
                            tc_mma_f16(tmem + 64u * b, smem_desc_sw128(a0 + kb * 128 * 128) + 2 * kk,
                                       smem_desc_sw128(g0 + kb * kColTileY * 128) + 2 * kk, idesc, (kb | kk) != 0);
                    tc_commit(&tmem_full[b]);
                    tc_commit(&a_empty[b]);
                }
            }
            if (has_next && !same) {
                // frequency change: G and both buffers are free once job j's MMA completed
                failed = !mbar_wait(&a_empty[j & 1], (j >> 1) & 1, abort_s);
                if (named_barrier_or(1, 128, failed)) {
                    if (ptid == 0) fail_status(a.status, abort_s, 34);
                    break;
                }
                load_g(freq_of(j + 1));
                issue(j + 1);
            }
        }
        cp_async_wait<0>();
        if (ptid == 0) {
            tc_commit(drain);
            if (!mbar_wait(drain, 0, abort_s)) {
                volatile int dummy = 0;
                mbar_wait(drain, 0, &dummy);
            }
        }
    } else {
        // -------------------------------------------------------------- epilogue
        // D[n][y]: warp w holds rows 32w .. 32w+31.
        //   paired:   warp 0 P, 1 Q (theta), 2 P', 3 Q' (pi - theta), x = lane
        //   unpaired: warps 0-1 P (x = 32 (w & 1) + lane), warps 2-3 Q
        const uint32_t lane_base = (uint32_t)(32 * warp) << 16;
        for (int j = 0; j < njobs; ++j) {
            const ColItem w = col_item(a, blockIdx.x + j * gridDim.x);
            const TcUnitDev u = a.units[w.unit];
            const TcFreqDev f = a.freqs[u.s];
            const int x0 = w.x0, y0 = w.y0, b = j & 1;
            const bool paired = u.plane_b >= 0;
            const bool is_q = paired ? (warp & 1) : (warp >= 2);
            const int slot = paired ? (warp >> 1) : (warp & 1);
            // row phases: lane l holds rows y0 + l and y0 + 32 + l
            const float2 py0 = (y0 + lane < a.H) ? __ldg(&u.phy[y0 + lane]) : make_float2(0.f, 0.f);
            const float2 py1 = (y0 + 32 + lane < a.H) ? __ldg(&u.phy[y0 + 32 + lane]) : make_float2(0.f, 0.f);
            const bool failed = !mbar_wait(&tmem_full[b], (j >> 1) & 1, abort_s);
            if (named_barrier_or(2, 128, failed)) {
                if (tid == 0) fail_status(a.status, abort_s, 33);
                break;
            }
            tc_fence_after();
            const float unscale = f.unscale_col;
            const uint32_t tb = tmem + lane_base + 64u * b;
            if (is_q) {
#pragma unroll 1
                for (int c0 = 0; c0 < kColTileY; c0 += 16) {
                    float v[16];
                    tmem_ld16(tb + c0, v);
#pragma unroll
                    for (int jj = 0; jj < 16; ++jj) xch[(slot * kColTileY + c0 + jj) * 32 + lane] = v[jj] * unscale;
                }
            }
            named_barrier(2, 128);
            if (!is_q) {
                const int x = x0 + (paired ? lane : 32 * slot + lane);
                const int plane = paired ? (slot == 0 ? u.plane_a : u.plane_b) : u.plane_a;
                float2 *o = a.out + (int64_t)plane * a.plane + x;
#pragma unroll 1
                for (int c0 = 0; c0 < kColTileY; c0 += 16) {
                    float v[16];
                    tmem_ld16(tb + c0, v);
#pragma unroll
                    for (int jj = 0; jj < 16; ++jj) {
                        const int r = c0 + jj;
                        const float2 pyr = r < 32 ? py0 : py1;
                        const float tx = __shfl_sync(0xffffffffu, pyr.x, r & 31);
                        const float ty = __shfl_sync(0xffffffffu, pyr.y, r & 31);
                        const int yy = y0 + r;
                        if (x < a.W && yy < a.H) {
                            const float P = v[jj] * unscale;
                            const float Q = xch[(slot * kColTileY + r) * 32 + lane];
                            // Eq. 7-8 (theta) and Eq. 15-16 (pi - theta)
                            __stcs(o + (int64_t)yy * a.W, make_float2(fmaf(tx, P, ty * Q), fmaf(ty, P, -tx * Q)));
                        }
                    }
                }
            }
            tc_fence_before();
            named_barrier(2, 128);   // xch is free for the next job
            if (lane == 0) mbar_arrive(&tmem_empty[b]);
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0) tmem_dealloc(tmem, 128);
}

// Largest |f| of the image as float bits (non-negative floats order like their integers).
__global__ void k_absmax(const float *__restrict__ img, int64_t pitch, int H, int W, int *__restrict__ out)
{
    float m = 0.f;
    for (int y = blockIdx.y; y < H; y += gridDim.y)
        for (int x = blockIdx.x * blockDim.x + threadIdx.x; x < W; x += gridDim.x * blockDim.x)
            m = fmaxf(m, fabsf(__ldg(img + (int64_t)y * pitch + x)));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    __shared__ float wm[32];
    if ((threadIdx.x & 31) == 0) wm[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int i = 1; i < (int)(blockDim.x >> 5); ++i) m = fmaxf(m, wm[i]);
        atomicMax(out, __float_as_int(m));   // one atomic per block
    }
}

// ------------------------------------------------------------------------ Toeplitz B (FP64)
// M[j][k] = S(k - j - off) * 2^sB for |k - j - off| <= R, `rows` rows, K-major SW128, FP16.
__global__ void k_build_toeplitz(uint16_t *__restrict__ B, int rows, int K, int off, int R, double sigma, int sB)
{
    const int n = rows * K;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int j = i / K, k = i % K;
        const int d = k - j - off;
        double v = 0.0;
        if (d >= -R && d <= R) v = ldexp(exp(-(double)d * d / (2.0 * sigma * sigma)) / (2.5066282746310002 * sigma), sB);
        B[sw128_offset(rows, j, k) / 2] = __half_as_ushort(__float2half_rn((float)v));
    }
}

TcGeometry gabor_tc_geometry(int R)
{
    TcGeometry g;
    g.R = R;
    g.R8 = round_up(R, 8);
    g.Krow = round_up(kRowTileX + 2 * R, 64);
    g.Kcol = round_up(kColTileY + g.R8 + R, 64);
    g.PW = round_up(kRowTileX + 2 * R, 4);
    g.smem_rows = 1024 + row_smem(g.Krow, g.PW, kRowTileYMax / 2).total;
    g.smem_cols = 1024 + col_smem(g.Kcol).total;
    return g;
}

size_t gabor_tc_smem_rows(int Kmax, int PWmax, int TY) { return 1024 + row_smem(Kmax, PWmax, TY).total; }
size_t gabor_tc_smem_cols(int Kmax) { return 1024 + col_smem(Kmax).total; }

bool gabor_tc_supported(int R)
{
    const TcGeometry g = gabor_tc_geometry(R);
    return g.smem_rows <= (size_t)kSmemLimit && g.smem_cols <= (size_t)kSmemLimit;
}

int gabor_tc_row_tile_x() { return kRowTileX; }
int gabor_tc_row_tile_y(int Rmax)
{
    const TcGeometry g = gabor_tc_geometry(Rmax);
    return (1024 + row_smem(g.Krow, g.PW, kRowTileYMax).total <= (size_t)kSmemLimit) ? kRowTileYMax : kRowTileYMax / 2;
}
int gabor_tc_col_tile_y() { return kColTileY; }

cudaError_t build_gabor_tc_b(uint16_t *Brow, uint16_t *Bcol, int R, double sigma, int bf16, float *unscale,
                             cudaStream_t st)
{
    (void)bf16;
    const TcGeometry g = gabor_tc_geometry(R);
    // max S = S(0) = 1 / (sqrt(2 pi) sigma): scale into [0.5, 1)
    int e = 0;
    frexp(1.0 / (2.5066282746310002 * sigma), &e);
    const int sB = -e;
    *unscale = (float)ldexp(1.0, -sB);
    k_build_toeplitz<<<(kRowTileX * g.Krow + 255) / 256, 256, 0, st>>>(Brow, kRowTileX, g.Krow, R, R, sigma, sB);
    cudaError_t err = cudaGetLastError();
    if (err != cudaSuccess) return err;
    k_build_toeplitz<<<(kColTileY * g.Kcol + 255) / 256, 256, 0, st>>>(Bcol, kColTileY, g.Kcol, g.R8, R, sigma, sB);
    return cudaGetLastError();
}

cudaError_t gabor_tc_prepare()
{
    cudaError_t e = cudaFuncSetAttribute(k_gabor_tc_rows, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemLimit);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_gabor_tc_cols, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemLimit);
    return e;
}

cudaError_t launch_gabor_tc(const TcBankArgs &a, int sm_count, cudaStream_t st)
{
    const int n_row_items = a.nf * a.row_cnt, n_col_items = a.nf * a.col_cnt;
    const size_t smem_r = gabor_tc_smem_rows(a.row_kmax, a.row_pwmax, a.row_ty);
    const size_t smem_c = gabor_tc_smem_cols(a.col_kmax);
    cudaError_t e0 = cudaMemsetAsync(a.absmax, 0, sizeof(int), st);
    if (e0 != cudaSuccess) return e0;
    const dim3 ag(std::max(1, std::min(4, (a.W + 255) / 256)), std::max(1, std::min(a.H, 2 * sm_count)));
    k_absmax<<<ag, 256, 0, st>>>(a.img, a.pitch, a.H, a.W, a.absmax);
    e0 = cudaGetLastError();
    if (e0 != cudaSuccess) return e0;
    if (n_row_items > 0) {
        k_gabor_tc_rows<<<std::min(n_row_items, sm_count), 384, smem_r, st>>>(a);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    if (n_col_items > 0) {
        k_gabor_tc_cols<<<std::min(n_col_items, sm_count), 256, smem_c, st>>>(a);
        return cudaGetLastError();
    }
    return cudaSuccess;
}

}  // namespace gb
