// Tensor-core localized sliding DFT (K5): Eq. 17 of arXiv 1704.05231 computed as the dense
// contraction "window x Gaussian-weighted twiddle matrix" on tcgen05 tensor cores.
//
// For a tile of 128 consecutive pixels of one image row, with k = b * Mx + a indexing the
// Mx x My window and n = 2 * bin + {re, im} indexing the bins (u, v), v in [0, My/2]:
//
//   D[p][n] = sum_k A[p][k] B[n][k],  A[p][k] = f(x0 + p - Mx/2 + a, y - My/2 + b) * 2^sA
//                                      B[n][k] = {Re, Im} exp(-i 2 pi (u a / Mx + v b / My))
//                                                S(a - Mx/2) S(b - My/2) * 2^sB
//
// B (built once per plan in FP64 on the GPU, stored pre-swizzled) arrives by one bulk copy
// (cp.async.bulk) and stays resident in shared memory for the whole persistent CTA.  D
// accumulates in FP32 in tensor memory, in two passes of NP columns each (2 x 256 TMEM
// columns), and is read back by the epilogue warps, rescaled exactly by 2^-(sA+sB), and stored
// as complex64; bins with v > My/2 are filled from F_{u,v} = F*_{Mx-u, My-v} (Algorithm 2,
// last loop).  A (FP16 or BF16) comes one of two ways:
//
//   k_sdft_tc_tma  (Mx in {8, 16, 32, 64}, Mx * My a multiple of 64): by TMA boxes of the
//                  pixel-major row-unfolded image U that k_unfold writes (sA from the image's
//                  max |f|, k_absmax); 16 epilogue warps, one MMA thread, one TMA thread.
//   k_sdft_tc      (other windows): by im2col in shared memory from a staged FP32 patch (sA
//                  per tile); 8 epilogue warps (TMEM lanes 0-127 = the tile's pixels, two per
//                  lane quadrant), 4 producer warps, one MMA thread.
//
// Every mbarrier wait is bounded; on timeout the CTA records a code in the status word and
// stops.
#include <algorithm>
#include <type_traits>

#include <cuda_fp16.h>
#include <cuda_bf16.h>

#include "internal.h"
#include "tc_common.cuh"

namespace gb {

namespace {

constexpr int kTileP = 128;   // pixels per tile (MMA M)

struct TcLayout {
    uint32_t b_off, a_off, patch_off, koff_off, bar_off, misc_off, total;
};

__host__ __device__ inline TcLayout tc_layout(int Kp, int NP, int My, int PW)
{
    TcLayout L;
    L.b_off = 0;
    L.a_off = L.b_off + (uint32_t)(Kp / 64) * (2 * NP) * 128;
    L.patch_off = L.a_off + (uint32_t)(Kp / 64) * kTileP * 128;
    L.koff_off = L.patch_off + (uint32_t)My * PW * 4;
    L.bar_off = (L.koff_off + (uint32_t)Kp * 4 + 15) & ~15u;
    L.misc_off = L.bar_off + 16 * 8;
    L.total = L.misc_off + 64;
    return L;
}

// Records the first failure code in the status word and raises the CTA's stop flag.
__device__ __forceinline__ void sdft_fail(int *status, volatile int *flag, int code)
{
    *flag = 1;
    atomicCAS(status, 0, code);
}

template <typename T> __device__ __forceinline__ uint16_t to_bits(float v);
template <> __device__ __forceinline__ uint16_t to_bits<__half>(float v) { return __half_as_ushort(__float2half_rn(v)); }
template <> __device__ __forceinline__ uint16_t to_bits<__nv_bfloat16>(float v)
{
    return __bfloat16_as_ushort(__float2bfloat16_rn(v));
}

}  // namespace

struct SdftTcArgs {
    CUtensorMap tmU;       // TMA-fed kernel: the row-unfolded image U (see k_unfold)
    const unsigned *maxbits;   // TMA-fed kernel: bits of max |f| (the scale of U)
    const float *img;
    int64_t pitch;
    int H, W;
    float2 *out;
    int64_t plane;
    int Mx, My, half;
    int K, Kp, NP, nbins, PW;
    const uint4 *Bglob;    // pre-swizzled B, b_bytes
    int b_bytes;
    float b_unscale;       // 2^-sB
    int tiles_x, ntiles;
    int *status;
    int bmode;             // BoundaryMode of the image beyond its edges
};

// Epilogue of both kernels (warps 0 .. 4 ngrp - 1): warp w reads TMEM lanes 32 (w % 4) .. +31
// (its pixels).  The 16-column chunks of a pass (8 bins each) are split among the quadrant's
// ngrp warps into contiguous ranges of equal store count (a bin with a mirrored partner costs
// two stores).  unscale_of(i, u) waits for tile i's operand scale and sets u = 2^-(sA + sB).
template <typename UnscaleFn>
__device__ __forceinline__ void sdft_tc_epilogue(const SdftTcArgs &a, uint32_t tmem, uint64_t *tmem_full,
                                                 uint64_t *tmem_empty, volatile int *abort_s, int ntiles_cta,
                                                 int warp, int lane, int ngrp, UnscaleFn unscale_of)
{
    const uint32_t lane_base = (uint32_t)(32 * (warp & 3)) << 16;
    const int cgrp = warp >> 2;
    const int nch = a.NP / 16;
    auto chunk_cost = [&](int h, int c) {
        const int bin0 = (h * a.NP + 16 * c) >> 1;
        if (bin0 >= a.nbins) return 0;
        const int v = bin0 / a.Mx;   // the chunk's first bin (a chunk may straddle two v)
        return (!a.half && v > 0 && 2 * v < a.My) ? 2 : 1;
    };
    // chunk c goes to group floor(ngrp x (cost of the chunks before c) / total)
    auto range_of = [&](int h, int &cb, int &ce) {
        int total = 0;
        for (int c = 0; c < nch; ++c) total += chunk_cost(h, c);
        cb = ce = nch;
        for (int c = 0, acc = 0; c < nch; acc += chunk_cost(h, c), ++c) {
            const int g = total > 0 ? acc * ngrp / total : 0;
            if (g == cgrp && cb == nch) cb = c;
            if (g > cgrp) { ce = c; break; }
        }
        if (cb > ce) cb = ce;
    };
    int cb0, ce0, cb1, ce1;
    range_of(0, cb0, ce0);
    range_of(1, cb1, ce1);
    const bool fast = a.Mx % 8 == 0;   // a chunk's 8 bins share v; nbins % 8 == 0
    for (int i = 0; i < ntiles_cta; ++i) {
        const int t = blockIdx.x + i * gridDim.x;
        const int y = t / a.tiles_x, x = (t % a.tiles_x) * kTileP + 32 * (warp & 3) + lane;
        float unscale = 0.f;
        bool ok = true;
        for (int h = 0; h < 2; ++h) {
            if (!mbar_wait(&tmem_full[h], i & 1, abort_s)) { ok = false; break; }
            if (h == 0 && !unscale_of(i, unscale)) { ok = false; break; }
            tc_fence_after();
            float2 *base = a.out + (int64_t)y * a.W + x;
            // Store the 8 bins of chunk c (accumulator columns 16 c .. + 15 of pass h).
            auto emit = [&](const uint32_t (&r)[16], int c) {
                if (x >= a.W) return;
                const int bin0 = (h * a.NP + 16 * c) >> 1;
                if (fast) {
                    if (bin0 >= a.nbins) return;
                    const int vv = bin0 / a.Mx, u0 = bin0 - vv * a.Mx;
                    float2 *pd = base + (int64_t)bin0 * a.plane;
#pragma unroll
                    for (int j = 0; j < 8; ++j)
                        __stcs(pd + j * a.plane, make_float2(__uint_as_float(r[2 * j]) * unscale,
                                                             __uint_as_float(r[2 * j + 1]) * unscale));
                    if (!a.half && vv > 0 && 2 * vv < a.My) {
                        // F_{Mx-u, My-v} = conj F_{u,v}: bins (My - vv) Mx + (Mx - u) mod Mx
                        float2 *pm = base + (int64_t)((a.My - vv) * a.Mx + a.Mx - u0) * a.plane;
                        float2 *p0 = u0 == 0 ? base + (int64_t)((a.My - vv) * a.Mx) * a.plane : pm;
                        __stcs(p0, make_float2(__uint_as_float(r[0]) * unscale, -__uint_as_float(r[1]) * unscale));
#pragma unroll
                        for (int j = 1; j < 8; ++j)
                            __stcs(pm - j * a.plane, make_float2(__uint_as_float(r[2 * j]) * unscale,
                                                                 -__uint_as_float(r[2 * j + 1]) * unscale));
                    }
                    return;
                }
                int vv = bin0 / a.Mx, uu = bin0 - vv * a.Mx;
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const int bin = bin0 + j;
                    if (bin < a.nbins) {
                        const float2 F = make_float2(__uint_as_float(r[2 * j]) * unscale,
                                                     __uint_as_float(r[2 * j + 1]) * unscale);
                        __stcs(base + (int64_t)bin * a.plane, F);
                        if (!a.half && vv > 0 && 2 * vv < a.My) {
                            const int um = uu == 0 ? 0 : a.Mx - uu;
                            __stcs(base + (int64_t)((a.My - vv) * a.Mx + um) * a.plane, make_float2(F.x, -F.y));
                        }
                    }
                    if (++uu == a.Mx) { uu = 0; ++vv; }
                }
            };
            // Ping-pong register buffers: the next chunk's TMEM load is in flight while the
            // current chunk is stored.
            const uint32_t tb = tmem + lane_base + 256u * h;
            uint32_t ra[16], rb[16];
            int c = h == 0 ? cb0 : cb1;
            const int ce = h == 0 ? ce0 : ce1;
            if (c < ce) {
                tmem_ld16_async(tb + 16 * c, ra);
                tmem_wait_ld();
            }
            while (c < ce) {
                if (c + 1 < ce) tmem_ld16_async(tb + 16 * (c + 1), rb);
                emit(ra, c);
                tmem_wait_ld();
                if (++c >= ce) break;
                if (c + 1 < ce) tmem_ld16_async(tb + 16 * (c + 1), ra);
                emit(rb, c);
                tmem_wait_ld();
                ++c;
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&tmem_empty[h]);
        }
        if (!ok) {
            if (lane == 0) { *abort_s = 1; atomicExch(a.status, 1); }
            break;
        }
    }
}

// EXT: a non-zero boundary rule (compile-time, so the zero rule keeps its lean load path).
template <typename T, bool EXT>
__global__ void __launch_bounds__(384, 1) k_sdft_tc(const SdftTcArgs a)
{
    extern __shared__ unsigned char smem_dyn[];
    unsigned char *sm = reinterpret_cast<unsigned char *>(((uintptr_t)smem_dyn + 1023) & ~(uintptr_t)1023);
    const TcLayout L = tc_layout(a.Kp, a.NP, a.My, a.PW);
    unsigned char *sB = sm + L.b_off;
    unsigned char *sA = sm + L.a_off;
    float *patch = reinterpret_cast<float *>(sm + L.patch_off);
    int *koff = reinterpret_cast<int *>(sm + L.koff_off);
    uint64_t *bars = reinterpret_cast<uint64_t *>(sm + L.bar_off);
    uint64_t *tmem_full = bars;        // [2]  MMA pass h done          (commit, count 1)
    uint64_t *tmem_empty = bars + 2;   // [2]  epilogue read pass h     (8 warps)
    uint64_t *a_empty = bars + 4;      // [1]  all MMAs of a tile done  (commit, count 1)
    uint64_t *scale_full = bars + 5;   // [2]  tile scale published     (count 1)
    uint64_t *final_bar = bars + 7;    // [1]  drain                    (commit, count 1)
    uint64_t *b_full = bars + 8;       // [1]  B landed                 (bulk copy)
    uint32_t *tmem_base_s = reinterpret_cast<uint32_t *>(sm + L.misc_off);
    volatile int *abort_s = reinterpret_cast<volatile int *>(sm + L.misc_off + 4);
    int *escale = reinterpret_cast<int *>(sm + L.misc_off + 8);        // [2]
    float *pmax = reinterpret_cast<float *>(sm + L.misc_off + 16);      // [4]

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    for (int k = tid; k < a.Kp; k += 384) {
        const int b = k / a.Mx, aa = k % a.Mx;
        koff[k] = k < a.K ? b * a.PW + aa : -1;
    }
    if (tid == 0) {
        mbar_init(&tmem_full[0], 1);
        mbar_init(&tmem_full[1], 1);
        mbar_init(&tmem_empty[0], 8);
        mbar_init(&tmem_empty[1], 8);
        mbar_init(a_empty, 1);
        mbar_init(&scale_full[0], 1);
        mbar_init(&scale_full[1], 1);
        mbar_init(final_bar, 1);
        mbar_init(b_full, 1);
        *abort_s = 0;
        mbar_fence_init();
        // B: resident for the whole CTA, one bulk copy that the first MMA waits for
        mbar_arrive_expect_tx(b_full, (uint32_t)a.b_bytes);
        bulk_load(smem_u32(sB), a.Bglob, (uint32_t)a.b_bytes, b_full);
    }
    if (warp == 0) {
        tmem_alloc(tmem_base_s, 512);
        tmem_relinquish();
    }
    fence_proxy_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_base_s;

    const int ntiles_cta = a.ntiles > (int)blockIdx.x ? (a.ntiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
    const int PWn = kTileP + a.Mx - 1;
    const uint32_t idesc = idesc_f16(std::is_same<T, __nv_bfloat16>::value ? 1 : 0, kTileP, a.NP);

    if (warp >= 8) {
        // ------------------------------------------------------------ producers
        const int ptid = tid - 256;
        bool b_landed = false;   // ptid 0: B's bulk copy waited for
        // The next tile's patch is prefetched into registers (kPre per thread) while the
        // current tile is converted, so its global-load latency is hidden.
        constexpr int kPre = 24;
        const int npatch = a.My * PWn;
        const bool prefetch = npatch <= 128 * kPre;
        float pre[kPre];
        auto load_patch = [&](int t) {
            const int y = t / a.tiles_x, x0 = (t % a.tiles_x) * kTileP;
            int b = 0, c = ptid;   // idx = ptid + 128 q = b * PWn + c, PWn > 128
#pragma unroll
            for (int q = 0; q < kPre; ++q) {
                float v = 0.f;
                if (b < a.My) {
                    const int gy = y - a.My / 2 + b, gx = x0 - a.Mx / 2 + c;
                    if (!EXT) {
                        if (gy >= 0 && gy < a.H && gx >= 0 && gx < a.W) v = __ldg(a.img + (int64_t)gy * a.pitch + gx);
                    } else {
                        v = __ldg(a.img + (int64_t)ext_coord(gy, a.H, a.bmode) * a.pitch + ext_coord(gx, a.W, a.bmode));
                    }
                }
                pre[q] = v;
                c += 128;
                if (c >= PWn) { c -= PWn; ++b; }
            }
        };
        if (prefetch && ntiles_cta > 0) load_patch(blockIdx.x);
        for (int i = 0; i < ntiles_cta; ++i) {
            // One collective decision per tile: stop if any role gave up.
            if (named_barrier_or(1, 128, *abort_s != 0)) break;
            const int t = blockIdx.x + i * gridDim.x;
            const int y = t / a.tiles_x, x0 = (t % a.tiles_x) * kTileP;
            // patch rows y - My/2 + b, columns x0 - Mx/2 + c (zero outside the image)
            float m = 0.f;
            if (prefetch) {
                int b = 0, c = ptid;
#pragma unroll
                for (int q = 0; q < kPre; ++q) {
                    if (b < a.My) {
                        patch[b * a.PW + c] = pre[q];
                        m = fmaxf(m, fabsf(pre[q]));
                    }
                    c += 128;
                    if (c >= PWn) { c -= PWn; ++b; }
                }
                if (i + 1 < ntiles_cta) load_patch(t + gridDim.x);
            } else {
                for (int idx = ptid; idx < npatch; idx += 128) {
                    const int b = idx / PWn, c = idx - b * PWn;
                    const int gy = y - a.My / 2 + b, gx = x0 - a.Mx / 2 + c;
                    float v = 0.f;
                    if (!EXT) {
                        if (gy >= 0 && gy < a.H && gx >= 0 && gx < a.W) v = __ldg(a.img + (int64_t)gy * a.pitch + gx);
                    } else {
                        v = __ldg(a.img + (int64_t)ext_coord(gy, a.H, a.bmode) * a.pitch + ext_coord(gx, a.W, a.bmode));
                    }
                    patch[b * a.PW + c] = v;
                    m = fmaxf(m, fabsf(v));
                }
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
            if (lane == 0) pmax[warp - 8] = m;
            // A must no longer be read by the previous tile's MMAs.
            bool failed = i > 0 && !mbar_wait(a_empty, (i - 1) & 1, abort_s);
            if (named_barrier_or(1, 128, failed)) {
                if (ptid == 0) { *abort_s = 1; atomicExch(a.status, 2); }
                break;
            }
            const float mx = fmaxf(fmaxf(pmax[0], pmax[1]), fmaxf(pmax[2], pmax[3]));
            int e = 0;
            if (mx > 0.f) frexpf(mx, &e);       // mx = f * 2^e, f in [0.5, 1)
            const float sc = ldexpf(1.f, -e);   // patch * sc in [-1, 1)
            if (a.Mx % 8 == 0 && a.K == a.Kp) {
                // Fast path: thread = pixel p; chunk kc holds a = a0 .. a0 + 7 of window row b.
                const int p = ptid;
                int b = 0, a0 = 0;
#pragma unroll 4
                for (int kc = 0; kc < a.Kp / 8; ++kc) {
                    const float *src = patch + b * a.PW + a0 + p;
                    uint32_t w[4];
#pragma unroll
                    for (int q = 0; q < 4; ++q)
                        w[q] = (uint32_t)to_bits<T>(src[2 * q] * sc) | ((uint32_t)to_bits<T>(src[2 * q + 1] * sc) << 16);
                    *reinterpret_cast<uint4 *>(sA + sw128_offset(kTileP, p, 8 * kc)) = make_uint4(w[0], w[1], w[2], w[3]);
                    a0 += 8;
                    if (a0 == a.Mx) { a0 = 0; ++b; }
                }
            } else {
                const int nchunk = kTileP * (a.Kp / 8);
                for (int cidx = ptid; cidx < nchunk; cidx += 128) {
                    const int p = cidx & (kTileP - 1), kc = cidx >> 7;
                    uint32_t w[4];
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const int o0 = koff[8 * kc + 2 * q], o1 = koff[8 * kc + 2 * q + 1];
                        const float v0 = o0 >= 0 ? patch[o0 + p] * sc : 0.f;
                        const float v1 = o1 >= 0 ? patch[o1 + p] * sc : 0.f;
                        w[q] = (uint32_t)to_bits<T>(v0) | ((uint32_t)to_bits<T>(v1) << 16);
                    }
                    *reinterpret_cast<uint4 *>(sA + sw128_offset(kTileP, p, 8 * kc)) = make_uint4(w[0], w[1], w[2], w[3]);
                }
            }
            fence_proxy_async_smem();
            if (ptid == 0) escale[i & 1] = e;
            named_barrier(1, 128);
            if (ptid == 0) {
                mbar_arrive(&scale_full[i & 1]);
                bool ok = true;
                if (!b_landed) {
                    b_landed = mbar_wait(b_full, 0, abort_s);
                    if (!b_landed) {
                        *abort_s = 1;
                        atomicExch(a.status, 4);
                        ok = false;
                    }
                }
                for (int h = 0; ok && h < 2; ++h) {
                    if (i > 0 && !mbar_wait(&tmem_empty[h], (i - 1) & 1, abort_s)) {
                        *abort_s = 1;
                        atomicExch(a.status, 3);
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t a0 = smem_u32(sA), b0 = smem_u32(sB) + (uint32_t)h * a.NP * 128;
                    for (int kb = 0; kb < a.Kp / 64; ++kb) {
#pragma unroll
                        for (int kk = 0; kk < 4; ++kk) {
                            const uint64_t ad = smem_desc_sw128(a0 + kb * kTileP * 128) + 2 * kk;
                            const uint64_t bd = smem_desc_sw128(b0 + kb * (2 * a.NP) * 128) + 2 * kk;
                            tc_mma_f16(tmem + 256u * h, ad, bd, idesc, (kb | kk) != 0);
                        }
                    }
                    tc_commit(&tmem_full[h]);
                }
                if (ok) tc_commit(a_empty);
            }
        }
        if (ptid == 0) {
            // Drain: every MMA this thread issued is complete before TMEM is released.
            tc_commit(final_bar);
            if (!mbar_wait(final_bar, 0, abort_s)) {
                // an abort was raised elsewhere or the MMAs never completed: wait once more
                volatile int dummy = 0;
                mbar_wait(final_bar, 0, &dummy);
            }
            if (!b_landed) {   // B's copy lands before shared memory is released
                volatile int dummy = 0;
                mbar_wait(b_full, 0, &dummy);
            }
        }
    } else {
        // ------------------------------------------------------------ epilogue
        sdft_tc_epilogue(a, tmem, tmem_full, tmem_empty, abort_s, ntiles_cta, warp, lane, 2, [&](int i, float &unscale) {
            if (!mbar_wait(&scale_full[i & 1], (i >> 1) & 1, abort_s)) return false;
            unscale = ldexpf(a.b_unscale, escale[i & 1]);
            return true;
        });
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0) tmem_dealloc(tmem, 512);
}

// ---------------------------------------------------------------- TMA-fed kernel
// For windows whose rows are a power-of-two fraction of a 64-element K-block (Mx in {8, 16, 32,
// 64}, Mx * My a multiple of 64) the A operand needs no im2col by threads: with the row-unfolded
// image U[x][r][a] = s f(x - Mx/2 + a, r - My/2) (FP16 / BF16, r in [0, H + My), the boundary
// rule applied; pixel-major, so the 64/Mx window rows of a K-block are 128 contiguous bytes of
// a pixel), K-block kb of the tile at (y, x0) is the 2-D box {64 values, 128 pixels} of U at
// ((y + kb 64/Mx) Mx, x0), which the TMA writes in the 128-byte-swizzled K-major layout.
// Roles (576 threads): warps 0-15 the epilogue above (4 per TMEM lane quadrant), warp 16 lane 0
// issues the MMAs, warp 17 lane 0 issues the TMA loads.  A is one buffer of Kp/64 K-blocks with
// a full / empty barrier pair each: K-block kb of the next tile is loaded as soon as the last
// MMA that reads it (pass 1) is done, so loads overlap the MMAs of later K-blocks and the
// epilogue.  The global scale s = 2^-e (max |f| = m 2^e, m in [0.5, 1)) comes with U.
constexpr int kTmaEpiWarps = 16;   // epilogue warps (4 per TMEM lane quadrant)
constexpr int kTmaThreads = 32 * (kTmaEpiWarps + 2);

__host__ __device__ inline TcLayout tc_layout_tma(int Kp, int NP)
{
    TcLayout L;
    L.b_off = 0;
    L.a_off = L.b_off + (uint32_t)(Kp / 64) * (2 * NP) * 128;
    L.patch_off = L.koff_off = L.a_off + (uint32_t)(Kp / 64) * kTileP * 128;
    L.bar_off = L.patch_off;
    L.misc_off = L.bar_off + 24 * 8;
    L.total = L.misc_off + 64;
    return L;
}

__device__ __forceinline__ int scale_exponent(unsigned maxbits)
{
    int e = 0;
    const float mx = __uint_as_float(maxbits);
    if (mx > 0.f) frexpf(mx, &e);   // mx = m * 2^e, m in [0.5, 1)
    return e;
}

template <typename T>
__global__ void __launch_bounds__(kTmaThreads, 1) k_sdft_tc_tma(const __grid_constant__ SdftTcArgs a)
{
    extern __shared__ unsigned char smem_dyn[];
    unsigned char *sm = reinterpret_cast<unsigned char *>(((uintptr_t)smem_dyn + 1023) & ~(uintptr_t)1023);
    const TcLayout L = tc_layout_tma(a.Kp, a.NP);
    unsigned char *sB = sm + L.b_off;
    unsigned char *sA = sm + L.a_off;
    uint64_t *bars = reinterpret_cast<uint64_t *>(sm + L.bar_off);
    uint64_t *tmem_full = bars;        // [2]  MMA pass h done                    (commit)
    uint64_t *tmem_empty = bars + 2;   // [2]  epilogue read pass h               (epilogue warps)
    uint64_t *final_bar = bars + 4;    // [1]  drain                              (commit)
    uint64_t *b_full = bars + 5;       // [1]  B landed                           (bulk copy)
    uint64_t *a_full = bars + 8;       // [4]  K-block kb of A landed             (TMA bytes)
    uint64_t *a_empty = bars + 12;     // [4]  the last MMA reading K-block kb done (commit)
    uint32_t *tmem_base_s = reinterpret_cast<uint32_t *>(sm + L.misc_off);
    volatile int *abort_s = reinterpret_cast<volatile int *>(sm + L.misc_off + 4);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int nkb = a.Kp / 64, rows_kb = 64 / a.Mx;
    if (tid == 0) {
        mbar_init(&tmem_full[0], 1);
        mbar_init(&tmem_full[1], 1);
        mbar_init(&tmem_empty[0], kTmaEpiWarps);
        mbar_init(&tmem_empty[1], kTmaEpiWarps);
        mbar_init(final_bar, 1);
        mbar_init(b_full, 1);
        for (int kb = 0; kb < nkb; ++kb) {
            mbar_init(&a_full[kb], 1);
            mbar_init(&a_empty[kb], 1);
        }
        *abort_s = 0;
        mbar_fence_init();
        mbar_arrive_expect_tx(b_full, (uint32_t)a.b_bytes);
        bulk_load(smem_u32(sB), a.Bglob, (uint32_t)a.b_bytes, b_full);
    }
    if (warp == 0) {
        tmem_alloc(tmem_base_s, 512);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    // Launched as a programmatic dependent of k_unfold: everything above (barriers, TMEM, the
    // copy of B) overlaps its tail; U and the scale are read only after it has completed.
    pdl_wait();
    const uint32_t tmem = *tmem_base_s;
    const int ntiles_cta = a.ntiles > (int)blockIdx.x ? (a.ntiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;

    if (warp == kTmaEpiWarps + 1) {
        // ------------------------------------------------------------ TMA producer (lane 0)
        if (lane == 0) {
            // K-block kb of tile i is loaded once the MMAs of tile i - 1 are done with it, so at
            // most one load per K-block is in flight; issued tiles: `full`, plus `part` K-blocks
            // of the tile where a wait gave up.
            int full = 0, part = 0;
            for (int i = 0; i < ntiles_cta && !*abort_s; ++i) {
                const int t = blockIdx.x + i * gridDim.x;
                const int y = t / a.tiles_x, x0 = (t % a.tiles_x) * kTileP;
                for (part = 0; part < nkb; ++part) {
                    if (i > 0 && !mbar_wait(&a_empty[part], (i - 1) & 1, abort_s)) {
                        sdft_fail(a.status, abort_s, 5);
                        break;
                    }
                    mbar_arrive_expect_tx(&a_full[part], 16384u);
                    tma_load_2d(smem_u32(sA) + part * 16384u, &a.tmU, (y + part * rows_kb) * a.Mx, x0, &a_full[part]);
                }
                if (part < nkb) break;
                full = i + 1;
                part = 0;
            }
            // Every load issued completes (consumed or not) before shared memory is released.
            for (int kb = 0; kb < nkb; ++kb) {
                const int n = full + (kb < part ? 1 : 0);
                if (n > 0) {
                    volatile int dummy = 0;
                    mbar_wait(&a_full[kb], (n - 1) & 1, &dummy);
                }
            }
        }
    } else if (warp == kTmaEpiWarps) {
        // ------------------------------------------------------------ MMA issuer (lane 0)
        if (lane == 0) {
            const uint32_t idesc = idesc_f16(std::is_same<T, __nv_bfloat16>::value ? 1 : 0, kTileP, a.NP);
            bool ok = mbar_wait(b_full, 0, abort_s);
            if (!ok) sdft_fail(a.status, abort_s, 6);
            for (int i = 0; ok && i < ntiles_cta; ++i) {
                for (int h = 0; ok && h < 2; ++h) {
                    if (i > 0 && !mbar_wait(&tmem_empty[h], (i - 1) & 1, abort_s)) {
                        sdft_fail(a.status, abort_s, 7);
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t a0 = smem_u32(sA), b0 = smem_u32(sB) + (uint32_t)h * a.NP * 128;
                    for (int kb = 0; kb < nkb; ++kb) {
                        if (h == 0 && !mbar_wait(&a_full[kb], i & 1, abort_s)) {
                            sdft_fail(a.status, abort_s, 8);
                            ok = false;
                            break;
                        }
                        tc_fence_after();
#pragma unroll
                        for (int kk = 0; kk < 4; ++kk) {
                            const uint64_t ad = smem_desc_sw128(a0 + kb * kTileP * 128) + 2 * kk;
                            const uint64_t bd = smem_desc_sw128(b0 + kb * (2 * a.NP) * 128) + 2 * kk;
                            tc_mma_f16(tmem + 256u * h, ad, bd, idesc, (kb | kk) != 0);
                        }
                        if (h == 1) tc_commit(&a_empty[kb]);
                    }
                    if (ok) tc_commit(&tmem_full[h]);
                }
            }
            // Drain: every MMA issued is complete before TMEM is released.
            tc_commit(final_bar);
            if (!mbar_wait(final_bar, 0, abort_s)) {
                volatile int dummy = 0;
                mbar_wait(final_bar, 0, &dummy);
            }
            if (!ok) {   // B's copy lands before shared memory is released
                volatile int dummy = 0;
                mbar_wait(b_full, 0, &dummy);
            }
        }
    } else {
        // ------------------------------------------------------------ epilogue
        const float unscale = ldexpf(a.b_unscale, scale_exponent(__ldg(a.maxbits)));
        sdft_tc_epilogue(a, tmem, tmem_full, tmem_empty, abort_s, ntiles_cta, warp, lane, kTmaEpiWarps / 4,
                         [&](int, float &u) {
            u = unscale;
            return true;
        });
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0) tmem_dealloc(tmem, 512);
}

// max |f| over the image, as float bits (non-negative floats order as unsigned integers); one
// atomic per block (256 threads)
__global__ void k_absmax(const float *__restrict__ img, int64_t pitch, int H, int W, unsigned *maxbits)
{
    pdl_launch_dependents();   // k_unfold may launch now (it waits for this grid before reading the max)
    __shared__ float wmax[8];
    float m = 0.f;
    const int64_t ystep = (int64_t)gridDim.y * pitch;
    for (int x = blockIdx.x * blockDim.x + threadIdx.x; x < W; x += gridDim.x * blockDim.x) {
        int y = blockIdx.y;
        // four rows' loads in flight per thread
        for (; y + 3 * (int)gridDim.y < H; y += 4 * (int)gridDim.y) {
            const float *p = img + (int64_t)y * pitch + x;
            const float v0 = __ldg(p), v1 = __ldg(p + ystep), v2 = __ldg(p + 2 * ystep), v3 = __ldg(p + 3 * ystep);
            m = fmaxf(m, fmaxf(fmaxf(fabsf(v0), fabsf(v1)), fmaxf(fabsf(v2), fabsf(v3))));
        }
        for (; y < H; y += gridDim.y) m = fmaxf(m, fabsf(__ldg(img + (int64_t)y * pitch + x)));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) wmax[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < 8; ++w) m = fmaxf(m, wmax[w]);
        if (m > 0.f) atomicMax(maxbits, __float_as_uint(m));
    }
}

// U[x][r][a] = s f(x - Mx/2 + a, r - My/2) for x in [0, W), r in [0, H + My), a in [0, Mx),
// the image extended by the boundary rule; one thread per (x, r), x fastest (a warp's loads of
// one image row are contiguous), Mx / 8 16-byte stores of its own 2 Mx bytes.
template <typename T>
__global__ void k_unfold(const float *__restrict__ img, int64_t pitch, int H, int W, int Mx, int My, int bmode,
                         const unsigned *maxbits, uint4 *__restrict__ U)
{
    // the SDFT kernel that reads U may start its prologue now (it waits for this grid's end);
    // this grid is itself a programmatic dependent of k_absmax
    pdl_launch_dependents();
    pdl_wait();
    const float sc = ldexpf(1.f, -scale_exponent(__ldg(maxbits)));
    const int64_t n = (int64_t)(H + My) * W;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int r = (int)(i / W), x = (int)(i - (int64_t)r * W);
        const int64_t o = ((int64_t)x * (H + My) + r) * Mx;   // U[x][r][0]
        const int gy = r - My / 2;
        const bool yin = gy >= 0 && gy < H;
        const float *row = img + (int64_t)(bmode == kBoundaryZero ? (yin ? gy : 0) : ext_coord(gy, H, bmode)) * pitch;
        const bool zrow = bmode == kBoundaryZero && !yin;
        for (int a0 = 0; a0 < Mx; a0 += 8) {
            uint32_t w[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                float v[2];
#pragma unroll
                for (int j = 0; j < 2; ++j) {
                    const int gx = x - Mx / 2 + a0 + 2 * q + j;
                    if (bmode == kBoundaryZero)
                        v[j] = (!zrow && gx >= 0 && gx < W) ? __ldg(row + gx) : 0.f;
                    else
                        v[j] = __ldg(row + ext_coord(gx, W, bmode));
                }
                w[q] = (uint32_t)to_bits<T>(v[0] * sc) | ((uint32_t)to_bits<T>(v[1] * sc) << 16);
            }
            U[(o + a0) / 8] = make_uint4(w[0], w[1], w[2], w[3]);
        }
    }
}

// ---------------------------------------------------------------- B builder (FP64)
__global__ void k_build_sdft_b(uint16_t *__restrict__ B, int Mx, int My, int K, int Kp, int NP, int nbins,
                               double sigma, int sB, int bf16)
{
    const int rows = 2 * NP;
    const int n_el = rows * Kp;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n_el; i += gridDim.x * blockDim.x) {
        const int n = i / Kp, k = i % Kp;
        const int bin = n >> 1, comp = n & 1;
        double val = 0.0;
        if (k < K && bin < nbins) {
            const int b = k / Mx, aa = k % Mx;
            const int v = bin / Mx, u = bin % Mx;
            const int ra = (u * aa) % Mx, rb = (v * b) % My;
            double s, c;
            // exp(-i phi), phi = 2 pi (ra / Mx + rb / My)
            sincospi(2.0 * ((double)ra / Mx + (double)rb / My), &s, &c);
            const double da = aa - Mx / 2, db = b - My / 2;
            const double g = exp(-(da * da + db * db) / (2.0 * sigma * sigma)) / (2.0 * 3.141592653589793 * sigma * sigma);
            val = (comp == 0 ? c : -s) * g;
            val = ldexp(val, sB);
        }
        const float fv = (float)val;
        const uint16_t bits = bf16 ? __bfloat16_as_ushort(__float2bfloat16_rn(fv)) : __half_as_ushort(__float2half_rn(fv));
        B[sw128_offset(rows, n, k) / 2] = bits;
    }
}

bool sdft_tc_supported(int Mx, int My)
{
    if (sdft_tc_tma_ok(Mx, My)) return true;
    const int K = Mx * My;
    if (K > 256) return false;
    const int Kp = round_up_i(K, 64);
    const int nbins = (My / 2 + 1) * Mx;
    const int NP = round_up_i((2 * nbins + 1) / 2, 16);
    if (NP > 256) return false;
    const int PW = round_up_i(kTileP + Mx - 1, 4);
    const TcLayout L = tc_layout(Kp, NP, My, PW);
    return L.total + 1024 <= (uint32_t)kSmemLimit;
}

bool sdft_tc_tma_ok(int Mx, int My)
{
    const int K = Mx * My;
    if (!(Mx == 8 || Mx == 16 || Mx == 32 || Mx == 64) || K % 64 != 0 || K > 256) return false;
    const int nbins = (My / 2 + 1) * Mx;
    const int NP = round_up_i(nbins, 16);
    return NP <= 256 && tc_layout_tma(K, NP).total + 1024 <= (uint32_t)kSmemLimit;
}

int64_t sdft_tc_ws_bytes(int H, int W, int Mx, int My)
{
    return sdft_tc_tma_ok(Mx, My) ? 256 + (int64_t)(H + My) * W * Mx * 2 : 0;
}

cudaError_t sdft_tc_prepare()
{
    cudaError_t e0 = cudaFuncSetAttribute(k_sdft_tc_tma<__half>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemLimit);
    if (e0 == cudaSuccess)
        e0 = cudaFuncSetAttribute(k_sdft_tc_tma<__nv_bfloat16>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemLimit);
    if (e0 != cudaSuccess) return e0;
    cudaError_t e = cudaFuncSetAttribute(k_sdft_tc<__half, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemLimit);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_sdft_tc<__nv_bfloat16, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemLimit);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_sdft_tc<__half, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemLimit);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_sdft_tc<__nv_bfloat16, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemLimit);
    return e;
}

// Builds B for (sigma, Mx, My) into *Bdev (allocated by the caller with sdft_tc_b_bytes()).
int sdft_tc_b_bytes(int Mx, int My)
{
    const int K = Mx * My, Kp = round_up_i(K, 64);
    const int nbins = (My / 2 + 1) * Mx;
    const int NP = round_up_i((2 * nbins + 1) / 2, 16);
    return Kp * 2 * NP * 2;
}

cudaError_t build_sdft_tc_b(void *Bdev, double sigma, int Mx, int My, int bf16, float *b_unscale, cudaStream_t st)
{
    const int K = Mx * My, Kp = round_up_i(K, 64);
    const int nbins = (My / 2 + 1) * Mx;
    const int NP = round_up_i((2 * nbins + 1) / 2, 16);
    // max |B| = S(0)^2 = 1 / (2 pi sigma^2); scale it into [0.5, 1)
    const double mx = 1.0 / (2.0 * 3.141592653589793 * sigma * sigma);
    int e = 0;
    frexp(mx, &e);
    const int sB = -e;
    *b_unscale = (float)ldexp(1.0, -sB);
    const int n_el = 2 * NP * Kp;
    k_build_sdft_b<<<(n_el + 255) / 256, 256, 0, st>>>(static_cast<uint16_t *>(Bdev), Mx, My, K, Kp, NP, nbins, sigma,
                                                        sB, bf16);
    return cudaGetLastError();
}

cudaError_t launch_sdft_tc(const float *img, int64_t pitch, int H, int W, float2 *out, int Mx, int My, int half,
                           const void *Bdev, float b_unscale, int bf16, int bmode, int *status, int sm_count,
                           void *ws, cudaStream_t st)
{
    SdftTcArgs a{};
    a.bmode = bmode;
    a.img = img;
    a.pitch = pitch;
    a.H = H;
    a.W = W;
    a.out = out;
    a.plane = (int64_t)H * W;
    a.Mx = Mx;
    a.My = My;
    a.half = half;
    a.K = Mx * My;
    a.Kp = round_up_i(a.K, 64);
    a.nbins = (My / 2 + 1) * Mx;
    a.NP = round_up_i((2 * a.nbins + 1) / 2, 16);
    a.PW = round_up_i(kTileP + Mx - 1, 4);
    a.Bglob = static_cast<const uint4 *>(Bdev);
    a.b_bytes = a.Kp * 2 * a.NP * 2;
    a.b_unscale = b_unscale;
    a.tiles_x = (W + kTileP - 1) / kTileP;
    a.ntiles = a.tiles_x * H;
    a.status = status;
    if (ws && sdft_tc_tma_ok(Mx, My)) {
        // workspace: [0, 4) max |f| bits, [256, ...) the unfolded image U
        unsigned *maxbits = static_cast<unsigned *>(ws);
        uint4 *U = reinterpret_cast<uint4 *>(static_cast<char *>(ws) + 256);
        cudaError_t e = cudaMemsetAsync(maxbits, 0, sizeof(unsigned), st);
        if (e != cudaSuccess) return e;
        const dim3 ag(std::max(1, std::min(4, (W + 255) / 256)), std::max(1, std::min(H, 2 * sm_count)));
        k_absmax<<<ag, 256, 0, st>>>(img, pitch, H, W, maxbits);
        const int64_t n = (int64_t)(H + My) * W;
        const int ub = (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 16 * sm_count));
        e = bf16 ? launch_pdl(k_unfold<__nv_bfloat16>, dim3(ub), dim3(256), 0, st, img, pitch, H, W, Mx, My, bmode,
                              static_cast<const unsigned *>(maxbits), U)
                 : launch_pdl(k_unfold<__half>, dim3(ub), dim3(256), 0, st, img, pitch, H, W, Mx, My, bmode,
                              static_cast<const unsigned *>(maxbits), U);
        if (e != cudaSuccess) return e;
        // U as a 2-D tensor ((H + My) Mx values of a pixel, W pixels): boxes of 64 x 128 (one
        // K-block of A: 128 pixel rows of 128 bytes), 128-byte swizzle
        PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
        if (!enc) return cudaErrorNotSupported;
        const cuuint64_t dims[2] = {(cuuint64_t)(H + My) * Mx, (cuuint64_t)W};
        const cuuint64_t strides[1] = {(cuuint64_t)(H + My) * Mx * 2};
        const cuuint32_t box[2] = {64, (cuuint32_t)kTileP};
        const cuuint32_t elem[2] = {1, 1};
        const CUresult r = enc(&a.tmU, bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2, U,
                               dims, strides, box, elem, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                               CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
        a.maxbits = maxbits;
        const TcLayout LT = tc_layout_tma(a.Kp, a.NP);
        const size_t smem = std::max<size_t>(LT.total + 1024, 120 * 1024);
        const dim3 grid(std::min(a.ntiles, sm_count)), block(kTmaThreads);
        return bf16 ? launch_pdl(k_sdft_tc_tma<__nv_bfloat16>, grid, block, smem, st, a)
                    : launch_pdl(k_sdft_tc_tma<__half>, grid, block, smem, st, a);
    }
    const TcLayout L = tc_layout(a.Kp, a.NP, My, a.PW);
    // at least ~half the SM's shared memory, so one CTA (and one 512-column TMEM block) per SM
    const size_t smem = std::max<size_t>(L.total + 1024, 120 * 1024);
    const int grid = std::min(a.ntiles, sm_count);
    const bool ext = bmode != kBoundaryZero;
    if (bf16)
        (ext ? k_sdft_tc<__nv_bfloat16, true> : k_sdft_tc<__nv_bfloat16, false>)<<<grid, 384, smem, st>>>(a);
    else
        (ext ? k_sdft_tc<__half, true> : k_sdft_tc<__half, false>)<<<grid, 384, smem, st>>>(a);
    return cudaGetLastError();
}

}  // namespace gb
