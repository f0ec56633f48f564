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
//                  written as FP16 to an intermediate laid out [signal][y / 8][x][8]: a
//                  thread's 8 rows of one column are one 16-byte block and a warp's stores
//                  cover 32 consecutive blocks.
//   column kernel  D[(signal, x)][y] = sum_l Sig[(signal, x)][l] G[y][l],  G[y][l] = S(l - y - R8)
//                  -> P, Q, P', Q' (Eq. 9).  Epilogue: F = remodulation by (cos, sin)(w^s y)
//                  (Eq. 7-8, 15-16), complex64 stores with coalesced rows.
//
// Both kernels are persistent (one CTA per SM) and warp-specialised.  Row kernel: 12 producer
// warps stage the patch and build Dm in the 128-byte-swizzled K-major layout, one producer
// thread issues tcgen05.mma into one of two TMEM buffers, 4 epilogue warps read the
// accumulators with tcgen05.ld.  Column kernel: one producer warp brings the A operands by TMA
// (cp.async.bulk.tensor) into up to four buffers and issues the MMAs into four TMEM
// accumulators; 8 epilogue warps.  The frequency's Toeplitz operand (T, G) arrives by one bulk
// copy (cp.async.bulk) on an mbarrier.  Every mbarrier wait is bounded.
#include <algorithm>
#include <type_traits>

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "internal.h"
#include "conv_fp32.cuh"
#include "tc_common.cuh"

namespace gb {

namespace {

constexpr int kRowTileX = 128;   // row kernel: image columns per tile (MMA M)
constexpr int kRowTileYMax = 64; // row kernel: image rows per tile (64, or 32 for large radii; MMA N = 2 x rows)
constexpr int kColTileY = 64;    // column kernel: output rows per tile (MMA N)
constexpr int kRowEpiWarps = 4;  // row kernel: epilogue warps (one per TMEM lane quarter); the rest produce

// (lo, hi) rounded to FP16 in one 32-bit word, lo in the low half (one cvt.rn.f16x2.f32).
__device__ __forceinline__ uint32_t h2pack(float lo, float hi)
{
    const __half2 h = __floats2half2_rn(lo, hi);
    return *reinterpret_cast<const uint32_t *>(&h);
}

// BF16 hi + lo split of (a, b): hi words bf16(a), bf16(b) and lo words bf16(a - hi), bf16(b - hi).
__device__ __forceinline__ void b2split(float a, float b, uint32_t &hi, uint32_t &lo)
{
    const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    const float2 hf = __bfloat1622float2(h);
    const __nv_bfloat162 l = __floats2bfloat162_rn(a - hf.x, b - hf.y);
    hi = *reinterpret_cast<const uint32_t *>(&h);
    lo = *reinterpret_cast<const uint32_t *>(&l);
}

__device__ __forceinline__ void fail_status(int *status, volatile int *flag, int code)
{
    *flag = 1;
    atomicExch(status, code);
}

// Per-CTA copy of the plan's descriptors (frequency order, frequencies, units) when they fit.
constexpr int kDescMaxFreqs = 32, kDescMaxUnits = 128;
constexpr uint32_t kDescBytes = (kDescMaxFreqs * 4 + kDescMaxFreqs * sizeof(TcFreqDev) +
                                 kDescMaxUnits * sizeof(TcUnitDev) + 127) / 128 * 128;

struct RowSmem {
    uint32_t t_off, dm_off, patch_off, ph_off, desc_off, bar_off, misc_off, total;
};

__host__ __device__ inline RowSmem row_smem(int K, int PW, int TY)
{
    RowSmem L;
    L.t_off = 0;
    L.dm_off = L.t_off + (uint32_t)kRowTileX * K * 2;
    L.patch_off = L.dm_off + (uint32_t)(2 * TY) * K * 2;
    L.ph_off = L.patch_off + (uint32_t)TY * (round_up(PW, 8) + 4) * 4;
    L.desc_off = (L.ph_off + 2u * PW * 8 + 15) & ~15u;
    L.bar_off = L.desc_off + kDescBytes;
    L.misc_off = L.bar_off + 8 * 8;
    L.total = L.misc_off + 64;
    return L;
}

struct ColSmem {
    uint32_t g_off, a_off, xch_off, desc_off, bar_off, misc_off, total;
};

constexpr int kColMaxStages = 4;   // A-operand buffers of the column kernel (at most)
constexpr int kColAcc = 4;         // TMEM accumulators (64 columns each) of the column kernel

__host__ __device__ inline ColSmem col_smem(int K, int nst)
{
    ColSmem L;
    L.g_off = 0;
    L.a_off = L.g_off + (uint32_t)kColTileY * K * 2;
    L.xch_off = L.a_off + (uint32_t)nst * 128 * K * 2;
    L.desc_off = L.xch_off + 4u * kColTileY * 32 * 4;
    L.bar_off = L.desc_off + kDescBytes;
    L.misc_off = L.bar_off + 24 * 8;
    L.total = L.misc_off + 64;
    return L;
}

// A buffers of the column kernel for K: up to kColMaxStages as shared memory allows, at least
// 2 (0: does not fit).
__host__ __device__ inline int col_stages(int K)
{
    for (int n = kColMaxStages; n >= 2; --n)
        if (1024 + col_smem(K, n).total <= (uint32_t)kSmemLimit) return n;
    return 0;
}

}  // namespace

// ------------------------------------------------------------------------- work items
// Items are decoded from the image shape: per frequency (largest radius first), the row pass
// has row_cnt tiles (TY rows x 128 columns); the column pass has, per unit, col_ny tiles of
// 64 rows x 32 columns (paired units, listed first) or x 64 columns (unpaired units).
struct RowItem {
    int s, y0, x0;
    int img;     // image of a batch (0 for one image)
};
struct ColItem {
    int unit, x0, y0;
};
// The plan's descriptors as the kernel reads them: shared-memory copies when they fit.
struct TcDesc {
    const int *forder;
    const TcFreqDev *freqs;
    const TcUnitDev *units;
};
// Copies the descriptors into `smem` (kDescBytes) when the plan is small enough; every thread
// of the CTA calls it, and a barrier must follow before the copies are read.
__device__ __forceinline__ TcDesc load_desc(const TcBankArgs &a, unsigned char *smem)
{
    const int nu = a.nf * a.nu_f;
    if (a.nf > kDescMaxFreqs || nu > kDescMaxUnits) return TcDesc{a.forder, a.freqs, a.units};
    int *fo = reinterpret_cast<int *>(smem);
    TcFreqDev *fr = reinterpret_cast<TcFreqDev *>(smem + kDescMaxFreqs * 4);
    TcUnitDev *un = reinterpret_cast<TcUnitDev *>(smem + kDescMaxFreqs * 4 + kDescMaxFreqs * sizeof(TcFreqDev));
    const int nw_f = a.nf * (int)(sizeof(TcFreqDev) / 4), nw_u = nu * (int)(sizeof(TcUnitDev) / 4);
    for (int i = threadIdx.x; i < a.nf; i += blockDim.x) fo[i] = a.forder[i];
    for (int i = threadIdx.x; i < nw_f; i += blockDim.x)
        reinterpret_cast<int *>(fr)[i] = reinterpret_cast<const int *>(a.freqs)[i];
    for (int i = threadIdx.x; i < nw_u; i += blockDim.x)
        reinterpret_cast<int *>(un)[i] = reinterpret_cast<const int *>(a.units)[i];
    return TcDesc{fo, fr, un};
}
__device__ __forceinline__ RowItem row_item(const TcBankArgs &a, const TcDesc &d, int it)
{
    const int g = it / a.row_cnt, local = it - g * a.row_cnt;
    return RowItem{d.forder[g], a.row_y0 + (local / a.row_nx) * a.row_ty, (local % a.row_nx) * kRowTileX};
}
__device__ __forceinline__ ColItem col_item(const TcBankArgs &a, const TcDesc &d, int it)
{
    const int g = it / a.col_cnt;
    int local = it - g * a.col_cnt;
    const int u0 = d.freqs[d.forder[g]].u0;
    const int paired_items = a.np_f * a.col_ny * a.col_nx32;
    const bool paired = local < paired_items;
    if (!paired) local -= paired_items;
    const int nx = paired ? a.col_nx32 : a.col_nx64;
    const int per = a.col_ny * nx, q = local / per, r = local - q * per;
    return ColItem{u0 + (paired ? 0 : a.np_f) + q, (r % nx) * (paired ? 32 : 64), (r / nx) * kColTileY};
}

// Output element (plane p, row y, column x): plane-major out[p][y][x] or pixel-major out[y][x][p].
__device__ __forceinline__ int64_t tc_out_offset(const TcBankArgs &a, int p, int y, int x)
{
    const int64_t pix = (int64_t)y * a.W + x;
    return a.layout ? pix * a.nplanes + p : (int64_t)p * a.plane + pix;
}

// The image an item works on: the call's image, or image i of a batch (with its TMA map).
struct TcImgView {
    const float *img;
    int64_t pitch;
    int H, W;
    float2 *out;
    int64_t plane;
    uint16_t *sig;
    int64_t Hp;
    const float2 *onesA, *onesB;
    const uint16_t *corrA, *corrB;
    const CUtensorMap *tm;
    int Wq;
    const CUtensorMap *tmP;   // the row pass's operand image (p_tma)
};
__device__ __forceinline__ TcImgView tc_img(const TcBankArgs &a, int i)
{
    if (a.imgs) {
        const TcImgDev d = a.imgs[i];
        return TcImgView{d.img, d.pitch, d.H, d.W, d.out, d.plane, d.sig, d.Hp, d.onesA, d.onesB, d.corrA, d.corrB,
                         a.tmaps + i, d.Wq, a.tmaps + a.nimg + i};
    }
    return TcImgView{a.img, a.pitch, a.H, a.W, a.out, a.plane, a.sig, a.Hp, a.onesA, a.onesB, a.corrA, a.corrB,
                     &a.tmA[0], a.Wq, &a.tmA[1]};
}
__device__ __forceinline__ int64_t tc_out_offset(const TcBankArgs &a, const TcImgView &im, int p, int y, int x)
{
    const int64_t pix = (int64_t)y * im.W + x;
    return a.layout ? pix * a.nplanes + p : (int64_t)p * im.plane + pix;
}

// Order-preserving unsigned keys of floats (for atomic min / max over signed values).
__device__ __forceinline__ unsigned fkey(float f)
{
    const unsigned b = __float_as_uint(f);
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}
__device__ __forceinline__ float fkey_value(unsigned k)
{
    return __uint_as_float((k & 0x80000000u) ? (k & 0x7fffffffu) : ~k);
}

// The centre c = (min + max) / 2 the passes subtract from the image, and e with
// max|f - c| = m 2^e, m in [0.5, 1) (FP16 operands get the exact scale 2^-e), from the
// order-preserving keys ~min, max.
__device__ __forceinline__ void centre_of(unsigned nlo, unsigned hik, float &c, int &e)
{
    const float lo = fkey_value(~nlo), hi = fkey_value(hik);
    c = hi >= lo ? 0.5f * (lo + hi) : 0.f;
    const float m = hi >= lo ? fmaxf(hi - c, c - lo) : 0.f;
    e = 0;
    if (m > 0.f) frexpf(m, &e);
}
__device__ __forceinline__ void image_centre(const TcBankArgs &a, float &c, int &e)
{
    centre_of(a.minmax[0], a.minmax[1], c, e);
}
// ... of image i: the call's image, or the per-image values k_ones wrote for a batch
__device__ __forceinline__ void tc_centre(const TcBankArgs &a, int i, float &c, int &e)
{
    if (a.img_ce) {
        const float2 v = a.img_ce[i];
        c = v.x;
        e = (int)v.y;
        return;
    }
    image_centre(a, c, e);
}

// ------------------------------------------------------------------------------ row pass
// Items: (frequency s, tile y, tile x), sorted by frequency; each item runs every unit of s.
// The image centre c and the scale 2^-e (|f - c| 2^-e < 1, FP16 range) come from k_minmax; the
// is applied to the staged patch after the image centre c is subtracted (the column pass adds
// c F[1] back).  Warps kRowEpiWarps .. 15 stage operands (the
// phases of the next unit arrive by cp.async while the current unit's operand is built);
// warps 0 .. kRowEpiWarps-1 are the epilogue (one or two per TMEM lane quarter).
__global__ void __launch_bounds__(512, 1) k_gabor_tc_rows(const __grid_constant__ TcBankArgs a)
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
    float *phbuf = reinterpret_cast<float *>(sm + L.ph_off);   // [2 slots][cos, sin][PWmax]
    uint64_t *bars = reinterpret_cast<uint64_t *>(sm + L.bar_off);
    uint64_t *tmem_full = bars;        // [2] commit
    uint64_t *tmem_empty = bars + 2;   // [2] 8 epilogue warps
    uint64_t *dm_empty = bars + 4;     // [1] commit: the MMA reading Dm is done
    uint64_t *drain = bars + 5;
    uint64_t *t_full = bars + 6;       // [1] T of a frequency landed (bulk copy)
    uint32_t *tmem_s = reinterpret_cast<uint32_t *>(sm + L.misc_off);
    volatile int *abort_s = reinterpret_cast<volatile int *>(sm + L.misc_off + 4);
    const TcDesc D = load_desc(a, sm + L.desc_off);

    if (tid == 0) {
        mbar_init(&tmem_full[0], 1);
        mbar_init(&tmem_full[1], 1);
        mbar_init(&tmem_empty[0], kRowEpiWarps);
        mbar_init(&tmem_empty[1], kRowEpiWarps);
        mbar_init(dm_empty, 1);
        mbar_init(drain, 1);
        mbar_init(t_full, 1);
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
    float cen;
    int e;
    image_centre(a, cen, e);

    if (warp >= kRowEpiWarps) {
        // -------------------------------------------------------------- producers
        constexpr int NP = 32 * (16 - kRowEpiWarps);   // producer threads
        const int ptid = tid - 32 * kRowEpiWarps, pwarp = warp - kRowEpiWarps;
        const float sc = ldexpf(1.f, -e);
        int cur_s = -1, job = 0;
        int t_loads = 0, t_landed = 0;   // T copies issued / waited for (uniform; ptid 0 waits)
        // cp.async of unit u's phases cos(w^c x), sin(w^c x) for the tile's columns into
        // phbuf[slot][0][.] and phbuf[slot][1][.]
        auto issue_phases = [&](const TcUnitDev &u, int x0, int R, int PW, int ncols, int slot) {
            float *dst = phbuf + slot * 2 * a.row_pwmax;
            const float *src = reinterpret_cast<const float *>(u.phx);
            for (int i = ptid; i < 2 * PW; i += NP) {
                const int c = i >> 1, cs = i & 1;
                const int gx = x0 - R + c;
                // beyond the image only for non-zero rules (extended samples keep their own phase)
                const bool ok = c < ncols && (a.bmode != kBoundaryZero || (gx >= 0 && gx < a.W));
                cp_async4(dst + cs * a.row_pwmax + c, ok ? (const void *)(src + 2 * gx + cs) : (const void *)src, ok ? 4 : 0);
            }
            cp_async_commit();
        };
        for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
            if (named_barrier_or(1, NP, *abort_s != 0)) break;
            const RowItem w = row_item(a, D, it);
            const int s = w.s, y0 = w.y0, x0 = w.x0;
            const TcFreqDev f = D.freqs[s];
            const int R = f.R, K = f.Krow;
            const int ncols = kRowTileX + 2 * R, PW = round_up(ncols, 4);
            const int PWs = round_up(PW, 8) + 4;     // row stride: 16-byte rows fall on distinct banks
            const int u0 = f.u0, nu = a.nu_f;
            // The previous item's last MMA (which read Dm, and T) must be complete.
            bool failed = job > 0 && !mbar_wait(dm_empty, (job - 1) & 1, abort_s);
            if (named_barrier_or(1, NP, failed)) {
                if (ptid == 0) fail_status(a.status, abort_s, 21);
                break;
            }
            if (s != cur_s) {
                // one bulk copy; the first MMA of the item waits for it
                if (ptid == 0) {
                    mbar_arrive_expect_tx(t_full, kRowTileX * K * 2);
                    bulk_load(smem_u32(sT), f.Brow, kRowTileX * K * 2, t_full);
                }
                ++t_loads;
                cur_s = s;
            }
            // patch rows y0 .. y0 + TY - 1, columns x0 - R .. x0 + 127 + R (zero outside the image)
            if (a.bmode == kBoundaryZero) {
                for (int r = pwarp; r < TY; r += NP / 32) {
                    const int y = y0 + r;
                    const bool yin = y >= 0 && y < a.H;
                    const float *src = a.img + (int64_t)(yin ? y : 0) * a.pitch;
                    for (int c = lane; c < PW; c += 32) {
                        const int gx = x0 - R + c;
                        const bool ok = yin && c < ncols && gx >= 0 && gx < a.W;
                        cp_async4(patch + r * PWs + c, ok ? (const void *)(src + gx) : (const void *)a.img, ok ? 4 : 0);
                    }
                }
            } else {
                for (int r = pwarp; r < TY; r += NP / 32) {
                    const float *src = a.img + (int64_t)ext_coord(y0 + r, a.H, a.bmode) * a.pitch;
                    for (int c = lane; c < PW; c += 32) {
                        const bool ok = c < ncols;
                        cp_async4(patch + r * PWs + c,
                                  ok ? (const void *)(src + ext_coord(x0 - R + c, a.W, a.bmode)) : (const void *)a.img,
                                  ok ? 4 : 0);
                    }
                }
            }
            cp_async_commit();
            issue_phases(D.units[u0], x0, R, PW, ncols, 0);
            cp_async_wait<0>();
            // (f - c) 2^-e on the thread's own patch elements; zero samples stay zero
            for (int r = pwarp; r < TY; r += NP / 32) {
                const int y = y0 + r;
                const bool yok = a.bmode != kBoundaryZero || (y >= 0 && y < a.H);
                for (int c = lane; c < PW; c += 32) {
                    const int gx = x0 - R + c;
                    const bool ok = yok && c < ncols && (a.bmode != kBoundaryZero || (gx >= 0 && gx < a.W));
                    patch[r * PWs + c] = ok ? (patch[r * PWs + c] - cen) * sc : 0.f;
                }
            }
            bool stop = false;
            for (int q = 0; q < nu; ++q, ++job) {
                const int b = job & 1;
                // Dm is read by the previous job's MMA.
                failed = q > 0 && !mbar_wait(dm_empty, (job - 1) & 1, abort_s);
                if (named_barrier_or(1, NP, failed)) {
                    if (ptid == 0) fail_status(a.status, abort_s, 22);
                    stop = true;
                    break;
                }
                // prefetch the next unit's phases (its buffer was read by job - 1's operand build)
                if (q + 1 < nu) {
                    issue_phases(D.units[u0 + q + 1], x0, R, PW, ncols, (q + 1) & 1);
                    cp_async_wait<1>();
                } else {
                    cp_async_wait<0>();
                }
                named_barrier(1, NP);    // this unit's phases (and the scaled patch) are visible
                // Dm[n = 2r + sg][k] = patch[r][k] (cos | sin)[k]: thread ptid keeps row
                // n = ptid mod 2TY and walks its 8-k chunks (broadcast phases, conflict-free
                // patch rows and swizzled stores).
                {
                    const int n = ptid % (2 * TY), r = n >> 1, sg = n & 1;
                    const float *prow = patch + r * PWs;
                    const float *phr = phbuf + ((q & 1) * 2 + sg) * a.row_pwmax;
                    const int kch = K / 8, kstep = NP / (2 * TY);
#pragma unroll 2
                    for (int kc = ptid / (2 * TY); kc < kch; kc += kstep) {
                        const int k0 = 8 * kc;
                        uint32_t wv[4];
                        if (k0 + 8 <= PW) {
                            const float4 p0 = *reinterpret_cast<const float4 *>(prow + k0);
                            const float4 p1 = *reinterpret_cast<const float4 *>(prow + k0 + 4);
                            const float4 h0 = *reinterpret_cast<const float4 *>(phr + k0);
                            const float4 h1 = *reinterpret_cast<const float4 *>(phr + k0 + 4);
                            wv[0] = h2pack(p0.x * h0.x, p0.y * h0.y);
                            wv[1] = h2pack(p0.z * h0.z, p0.w * h0.w);
                            wv[2] = h2pack(p1.x * h1.x, p1.y * h1.y);
                            wv[3] = h2pack(p1.z * h1.z, p1.w * h1.w);
                        } else {
                            float vv[8];
#pragma unroll
                            for (int t = 0; t < 8; ++t) vv[t] = (k0 + t < PW) ? prow[k0 + t] * phr[k0 + t] : 0.f;
#pragma unroll
                            for (int t = 0; t < 4; ++t) wv[t] = h2pack(vv[2 * t], vv[2 * t + 1]);
                        }
                        *reinterpret_cast<uint4 *>(sDm + sw128_offset(2 * TY, n, k0)) =
                            make_uint4(wv[0], wv[1], wv[2], wv[3]);
                    }
                }
                fence_proxy_async_smem();
                named_barrier(1, NP);
                if (ptid == 0) {
                    const bool t_ok = t_landed == t_loads || mbar_wait(t_full, (t_loads - 1) & 1, abort_s);
                    if (t_ok) t_landed = t_loads;
                    if (!t_ok) {
                        fail_status(a.status, abort_s, 25);
                    } else if (job >= 2 && !mbar_wait(&tmem_empty[b], ((job - 2) >> 1) & 1, abort_s)) {
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
        cp_async_wait<0>();
        if (ptid == 0) {
            tc_commit(drain);
            if (!mbar_wait(drain, 0, abort_s)) {
                volatile int dummy = 0;
                mbar_wait(drain, 0, &dummy);
            }
            if (t_landed < t_loads) {   // a copy still in flight after an abort lands first
                volatile int dummy = 0;
                mbar_wait(t_full, (t_loads - 1) & 1, &dummy);
            }
        }
    } else {
        // -------------------------------------------------------------- epilogue
        // Thread = image column x0 + x (TMEM lane x); accumulator columns 2r + {c, s}.  Warp
        // w reads lane quarter w & 3 and rows [rbase, rbase + rpw) of the tile.
        const int quarter = warp & 3, half = warp >> 2;
        const int x = 32 * quarter + lane;
        const uint32_t lane_base = (uint32_t)(32 * quarter) << 16;
        const int rpw = TY / (kRowEpiWarps / 4), rbase = half * rpw;
        int job = 0;
        for (int it = blockIdx.x; it < nitems && !*abort_s; it += gridDim.x) {
            const RowItem w = row_item(a, D, it);
            const int y0 = w.y0;
            const TcFreqDev f = D.freqs[w.s];
            const float unscale = ldexpf(f.unscale_row, e);
            const int gx = w.x0 + x;
            const bool xin = gx < a.W;
            const int u0 = f.u0, nu = a.nu_f;
            bool ok = true;
            for (int q = 0; q < nu; ++q, ++job) {
                const TcUnitDev u = D.units[u0 + q];
                const int b = job & 1;
                // row phases of the warp's rows: lane l holds rows rbase + l and rbase + 32 + l
                // (broadcast by shuffle)
                const int yl = y0 + rbase + lane, yl1 = yl + 32;
                const bool yok = a.bmode != kBoundaryZero || yl < a.H;
                const bool yok1 = a.bmode != kBoundaryZero || yl1 < a.H;
                const float2 pyl = (lane < rpw && yok) ? __ldg(&u.phy[yl]) : make_float2(0.f, 0.f);
                const float2 pyl1 = (lane + 32 < rpw && yok1) ? __ldg(&u.phy[yl1]) : make_float2(0.f, 0.f);
                const float2 px = xin ? __ldg(&u.phx[gx]) : make_float2(0.f, 0.f);
                if (!mbar_wait(&tmem_full[b], (job >> 1) & 1, abort_s)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const bool paired = u.plane_b >= 0;
                const int64_t sstride = (int64_t)a.W * a.Hp;   // between signals of the unit
                const int64_t bstride = (int64_t)a.W * 8;      // between 8-row blocks
                uint16_t *dst0 = a.sig + u.sig_idx * sstride + (int64_t)((a.Lpad + y0) >> 3) * bstride +
                                 (int64_t)(xin ? gx : 0) * 8;
#pragma unroll 1
                for (int c0 = 2 * rbase; c0 < 2 * (rbase + rpw); c0 += 16) {
                    float v[16];
                    tmem_ld16(tmem + lane_base + 128u * b + c0, v);
                    const int r0 = c0 >> 1;
                    uint32_t pk[4][4];
#pragma unroll
                    for (int jp = 0; jp < 4; ++jp) {
                        float sgl[2][4];
#pragma unroll
                        for (int t = 0; t < 2; ++t) {
                            const int j = 2 * jp + t;
                            const int rl = r0 + j - rbase;
                            const float2 pr = rl < 32 ? pyl : pyl1;
                            const float2 cy = make_float2(__shfl_sync(0xffffffffu, pr.x, rl & 31),
                                                          __shfl_sync(0xffffffffu, pr.y, rl & 31));
                            const float A = v[2 * j] * unscale, B = v[2 * j + 1] * unscale;
                            // Eq. 5-6: Re J = cos A + sin B, Im J = sin A - cos B
                            const float jr = fmaf(px.x, A, px.y * B), ji = fmaf(px.y, A, -px.x * B);
                            // Eq. 10
                            const float fcr = jr * cy.x, fsr = jr * cy.y, fci = ji * cy.x, fsi = ji * cy.y;
                            sgl[t][0] = fcr + fsi;
                            sgl[t][1] = fsr - fci;
                            sgl[t][2] = fcr - fsi;
                            sgl[t][3] = fsr + fci;
                        }
#pragma unroll
                        for (int g = 0; g < 4; ++g) pk[g][jp] = h2pack(sgl[0][g], sgl[1][g]);
                    }
                    if (xin) {
                        uint16_t *d = dst0 + (int64_t)(r0 >> 3) * bstride;   // lanes: consecutive 16-byte blocks
                        *reinterpret_cast<uint4 *>(d) = make_uint4(pk[0][0], pk[0][1], pk[0][2], pk[0][3]);
                        *reinterpret_cast<uint4 *>(d + sstride) = make_uint4(pk[1][0], pk[1][1], pk[1][2], pk[1][3]);
                        if (paired) {
                            *reinterpret_cast<uint4 *>(d + 2 * sstride) = make_uint4(pk[2][0], pk[2][1], pk[2][2], pk[2][3]);
                            *reinterpret_cast<uint4 *>(d + 3 * sstride) = make_uint4(pk[3][0], pk[3][1], pk[3][2], pk[3][3]);
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

// ------------------------------------------------------------ row pass, modulated taps
// GB_OPT_ROW_PASS = 2 (default): Eq. 5-6 as one product with a per-unit operand of modulated
// taps, no per-unit demodulated copy of the patch:
//
//   D[(x, re|im)][r] = sum_k Am[(x, re|im)][k] P[r][k],
//   Am[(x, re)][k] = S(d) cos(w^c d),  Am[(x, im)][k] = -S(d) sin(w^c d),  d = k - x - R8,
//   P[r][k] = (f(y0 + r, x0 - R8 + k) - c) 2^-e          (R8 = R rounded up to 8)
//
// -> Re J, Im J of 64 columns x TY rows of one unit (operand row n = 2 x + re|im).  Per item
// (frequency, tile): P once, either as TMA boxes of the operand image that k_ones wrote (zero
// rule; the window starts at x0 - R8, a multiple of 8 elements, as a tiled copy needs) or built
// by producer warps 8-14 from the image; the MMA thread brings each unit's Am (built once per
// plan) by one bulk copy into one of three buffers and issues the MMAs; 8 epilogue warps (two
// per lane quarter) store J itself, two signals per unit, for the modulated-tap column pass.
constexpr int kMtTileX = 64;     // output columns per item (MMA M = 2 x 64)
constexpr int kMtEpiWarps = 8;

// The modulated-tap operands are banded Toeplitz matrices with interleaved (re, im) rows:
// row n = 2 x + part, column k, value t_part(k - x - off).  With x counted backwards from the
// tile's last row, the no-swizzle K-major core matrix of 8-row group g and K-group kc holds
// t(4 (2 kc + g) + c + r / 2 - off') at (row r, element c): it depends on j = 2 kc + g only.
// So the operand is a strip of core matrices Q_j, 128 bytes each, read by one descriptor with
// 256 bytes between K-groups and 128 bytes between row groups; `rows` rows and K columns take
// 2 K / 8 + rows / 8 cores (instead of rows x K elements).
__host__ __device__ constexpr int tstrip_cores(int K, int rows) { return 2 * (K / 8) + rows / 8; }
__host__ __device__ constexpr uint32_t tstrip_bytes(int K, int rows) { return (uint32_t)tstrip_cores(K, rows) * 128u; }
// Descriptor of K step ks (16 columns) of a strip at shared address s0.
__device__ __forceinline__ uint64_t tstrip_desc(uint32_t s0, int ks) { return smem_desc_kmajor(s0 + 512u * ks, 256, 128); }

struct MtSmem {
    uint32_t a_off, p_off, patch_off, desc_off, bar_off, misc_off, total;
};
constexpr int kAmBufs = 3;   // Am strip buffers of the modulated-tap row kernel

// split = 1 (BF16 operands as hi + lo pairs): two strips per A buffer and P as hi and lo.
__host__ __device__ inline MtSmem mt_smem(int K, int PW, int TY, int split = 0)
{
    MtSmem L;
    const uint32_t np = split ? 2u : 1u;
    (void)PW;
    L.a_off = 0;                                              // [kAmBufs] buffers of np strips of 128 rows x K
    L.p_off = (L.a_off + kAmBufs * np * tstrip_bytes(K, 128) + 1023) & ~1023u;   // [2] x np x TY x K (SW128)
    L.patch_off = L.p_off + 2 * np * (uint32_t)TY * K * 2;
    L.desc_off = (L.patch_off + 127) & ~127u;
    L.bar_off = L.desc_off + kDescBytes;
    L.misc_off = L.bar_off + 16 * 8;
    L.total = L.misc_off + 64;
    return L;
}

__device__ __forceinline__ RowItem row_item_mt(const TcBankArgs &a, const TcDesc &d, int it)
{
    if (a.row_list) {
        const int4 v = a.row_list[it];
        return RowItem{v.y, v.z, v.w, v.x};
    }
    const int g = it / a.row_cnt, local = it - g * a.row_cnt;
    return RowItem{d.forder[g], a.row_y0 + (local / a.row_nx) * a.row_ty, (local % a.row_nx) * kMtTileX, 0};
}

// SPLIT: BF16 operands as hi + lo pairs (a.split); FP16 operands otherwise.
template <bool SPLIT>
__global__ void __launch_bounds__(512, 2) k_gabor_tc_rows_mt(const __grid_constant__ TcBankArgs a)
{
    const int nitems = a.row_list ? a.n_row : a.nf * a.row_cnt;
    extern __shared__ unsigned char smem_dyn[];
    unsigned char *sm = reinterpret_cast<unsigned char *>(((uintptr_t)smem_dyn + 1023) & ~(uintptr_t)1023);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int TY = a.row_ty;
    const MtSmem L = mt_smem(a.row_kmax, a.row_pwmax, TY, SPLIT ? 1 : 0);
    unsigned char *sA = sm + L.a_off;
    unsigned char *sP = sm + L.p_off;   // two P buffers (items alternate)
    uint64_t *bars = reinterpret_cast<uint64_t *>(sm + L.bar_off);
    uint64_t *tmem_full = bars;        // [2] commit
    uint64_t *tmem_empty = bars + 2;   // [2] epilogue warps
    uint64_t *a_full = bars + 4;       // [kAmBufs] Am landed (bulk copy)
    uint64_t *p_empty = bars + 4 + kAmBufs;   // [2] commit: the item's MMAs (reading P) are done
    uint64_t *drain = bars + 6 + kAmBufs;
    uint64_t *p_full = bars + 7 + kAmBufs;    // [2] the producers built the item's P
    uint32_t *tmem_s = reinterpret_cast<uint32_t *>(sm + L.misc_off);
    volatile int *abort_s = reinterpret_cast<volatile int *>(sm + L.misc_off + 4);
    volatile int *issued_s = reinterpret_cast<volatile int *>(sm + L.misc_off + 8);   // Am copies issued
    volatile int *landed_s = reinterpret_cast<volatile int *>(sm + L.misc_off + 12);  // Am copies waited for
    volatile int *p_issued_s = reinterpret_cast<volatile int *>(sm + L.misc_off + 16);  // P loads issued (TMA)
    volatile int *p_landed_s = reinterpret_cast<volatile int *>(sm + L.misc_off + 20);  // P loads waited for
    const TcDesc D = load_desc(a, sm + L.desc_off);
    constexpr uint32_t np = SPLIT ? 2u : 1u;
    const uint32_t abuf = np * tstrip_bytes(a.row_kmax, 128);   // an A buffer (hi, lo strips)
    const uint32_t plo = (uint32_t)TY * a.row_kmax * 2;         // P lo after P hi (split)
    const uint32_t pbuf = np * plo;                              // one P buffer (hi, lo)

    if (tid == 0) {
        for (int i = 0; i < 2; ++i) {
            mbar_init(&tmem_full[i], 1);
            mbar_init(&tmem_empty[i], kMtEpiWarps);
        }
        for (int i = 0; i < kAmBufs; ++i) mbar_init(&a_full[i], 1);
        for (int i = 0; i < 2; ++i) {
            mbar_init(&p_empty[i], 1);
            mbar_init(&p_full[i], 1);
        }
        mbar_init(drain, 1);
        *issued_s = 0;
        *landed_s = 0;
        *p_issued_s = 0;
        *p_landed_s = 0;
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
    // programmatic dependent of k_ones (which waits for k_minmax): the set-up above overlaps
    // them; the centre and scale are read after they completed
    pdl_launch_dependents();
    pdl_wait();
    const uint32_t tmem = *tmem_s;
    const uint32_t idesc = idesc_f16(SPLIT ? 1 : 0, 128, TY);
    const int my_items = (int)blockIdx.x < nitems ? (nitems - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
    const int njobs_row = my_items * a.nu_f;
    auto issue_am = [&](int jq) {   // the Am copy of job jq into buffer jq % kAmBufs
        const int buf = jq % kAmBufs;
        const RowItem w = row_item_mt(a, D, blockIdx.x + (jq / a.nu_f) * gridDim.x);
        const TcFreqDev f = D.freqs[w.s];
        const uint32_t abytes = np * tstrip_bytes(f.Kmt, 128);
        mbar_arrive_expect_tx(&a_full[buf], abytes);
        bulk_load(smem_u32(sA + buf * abuf), D.units[f.u0 + jq % a.nu_f].Am, abytes, &a_full[buf]);
    };

    if (warp == 15) {
        // -------------------------------------------------------------- MMA warp (lane 0)
        // The Am copy of job jq (unit jq % nu of the CTA's item jq / nu) goes into buffer
        // jq % kAmBufs: this warp issues the first kAmBufs; the others are issued by the epilogue
        // (warp 0) as soon as the MMAs of job jq - kAmBufs are complete.  The MMAs of an item wait
        // for its P (p_full) and release it (p_empty).
        if (lane == 0) {
            const int nu = a.nu_f;
            int landed = 0, p_landed = 0;
            bool ok = true;
            for (int jq = 0; jq < kAmBufs && jq < njobs_row; ++jq) issue_am(jq);
            for (int nitem = 0; nitem < my_items && ok; ++nitem) {
                const RowItem w = row_item_mt(a, D, blockIdx.x + nitem * gridDim.x);
                const int K = D.freqs[w.s].Kmt;
                const int pb = nitem & 1;
                if (ok) ok = mbar_wait(&p_full[pb], (nitem >> 1) & 1, abort_s);   // this item's P
                if (ok) p_landed = nitem + 1;
                for (int q = 0; q < nu && ok; ++q) {
                    const int jq = nitem * nu + q, b = jq & 1, ab = jq % kAmBufs;
                    ok = mbar_wait(&a_full[ab], (jq / kAmBufs) & 1, abort_s);
                    if (ok) landed = jq + 1;   // copy jq (copies go in job order)
                    if (ok && jq >= 2) ok = mbar_wait(&tmem_empty[b], ((jq - 2) >> 1) & 1, abort_s);
                    if (!ok) break;
                    tc_fence_after();
                    const uint32_t a0 = smem_u32(sA + ab * abuf), p0 = smem_u32(sP + pb * pbuf);
                    const uint32_t a0l = a0 + tstrip_bytes(K, 128);
                    for (int kb = 0; kb < K / 64; ++kb)
#pragma unroll
                        for (int kk = 0; kk < 4; ++kk) {
                            const uint64_t pd = smem_desc_sw128(p0 + kb * TY * 128) + 2 * kk;
                            tc_mma_f16(tmem + (uint32_t)TY * b, tstrip_desc(a0, 4 * kb + kk), pd, idesc, (kb | kk) != 0);
                            if constexpr (SPLIT) {   // Am_hi P_lo + Am_lo P_hi (the lo x lo product is dropped)
                                tc_mma_f16(tmem + (uint32_t)TY * b, tstrip_desc(a0, 4 * kb + kk),
                                           smem_desc_sw128(p0 + plo + kb * TY * 128) + 2 * kk, idesc, 1);
                                tc_mma_f16(tmem + (uint32_t)TY * b, tstrip_desc(a0l, 4 * kb + kk), pd, idesc, 1);
                            }
                        }
                    tc_commit(&tmem_full[b]);
                }
                if (ok) tc_commit(&p_empty[pb]);
            }
            if (!ok) fail_status(a.status, abort_s, 27);
            tc_commit(drain);
            if (!mbar_wait(drain, 0, abort_s)) {
                volatile int dummy = 0;
                mbar_wait(drain, 0, &dummy);
            }
            *landed_s = landed;
            *p_landed_s = p_landed;
        }
    } else if (warp >= kMtEpiWarps && a.p_tma) {
        // -------------------------------------------------------------- P by TMA (warp 8, lane 0)
        // The K / 64 boxes of 64 columns x TY rows (hi, then lo under split) of the operand image
        // at (x0 - R8 + 64 kb, y0) into buffer it & 1, once the MMAs of item it - 2 are done;
        // zeros outside the image, as the zero rule wants.
        if (warp == kMtEpiWarps && lane == 0) {
            int nitem = 0;
            for (int it = blockIdx.x; it < nitems && !*abort_s; it += gridDim.x, ++nitem) {
                const RowItem w = row_item_mt(a, D, it);
                const TcImgView im = tc_img(a, w.img);
                const TcFreqDev f = D.freqs[w.s];
                const int pb = nitem & 1, nkb = f.Kmt / 64;
                if (nitem < 2) prefetch_tmap(im.tmP);
                if (nitem >= 2 && !mbar_wait(&p_empty[pb], ((nitem - 2) >> 1) & 1, abort_s)) {
                    fail_status(a.status, abort_s, 26);
                    break;
                }
                mbar_arrive_expect_tx(&p_full[pb], np * (uint32_t)nkb * TY * 128u);
                const uint32_t dP = smem_u32(sP + pb * pbuf);
                for (uint32_t z = 0; z < np; ++z)
                    for (int kb = 0; kb < nkb; ++kb)
                        tma_load_3d(dP + z * plo + (uint32_t)kb * TY * 128u, im.tmP, w.x0 - f.R8 + 64 * kb, w.y0,
                                    (int)z, &p_full[pb]);
                *p_issued_s = nitem + 1;
            }
        }
    } else if (warp >= kMtEpiWarps) {
        // -------------------------------------------------------------- producers (warps 8-14)
        // P of item it into buffer it's parity, straight from the image: P[r][k] =
        // (f(x0 - R8 + k, y0 + r) - c) 2^-e in FP16 (zero beyond the window, and outside the image
        // under the zero rule), 8 k per 16-byte chunk of the swizzled K-major layout; a thread
        // takes chunks k8 = idx % (K / 8) of row r = idx / (K / 8), so a warp reads consecutive
        // 32-byte runs of image rows.  The buffer is free once the MMAs of item it - 2 are done.
        constexpr int NP = 32 * (15 - kMtEpiWarps);
        const int ptid = tid - 32 * kMtEpiWarps;
        int nitem = 0;
        for (int it = blockIdx.x; it < nitems; it += gridDim.x, ++nitem) {
            if (named_barrier_or(1, NP, *abort_s != 0)) break;
            const RowItem w = row_item_mt(a, D, it);
            const int y0 = w.y0, x0 = w.x0;
            const TcImgView im = tc_img(a, w.img);
            float cen;
            int e;
            tc_centre(a, w.img, cen, e);
            const float sc = ldexpf(1.f, -e);
            const TcFreqDev f = D.freqs[w.s];
            const int R = f.R, R8 = f.R8, K = f.Kmt, nk8 = K / 8;
            const int ncols = kMtTileX + R8 + R;
            const int pb = nitem & 1;
            bool failed = nitem >= 2 && !mbar_wait(&p_empty[pb], ((nitem - 2) >> 1) & 1, abort_s);
            if (named_barrier_or(1, NP, failed)) {
                if (ptid == 0) fail_status(a.status, abort_s, 26);
                break;
            }
            unsigned char *dP = sP + pb * pbuf;
            const bool zero = a.bmode == kBoundaryZero;
            const int nchunks = TY * nk8;
            // the loads of kU chunks are issued before any of them is converted
            constexpr int kU = 2;
            for (int base = ptid; base < nchunks; base += kU * NP) {
                float v[kU][8];
#pragma unroll
                for (int uu = 0; uu < kU; ++uu) {
                    const int idx = base + uu * NP;
                    const int r = idx / nk8, k0 = 8 * (idx - r * nk8);
                    const int y = y0 + r, gx0 = x0 - R8 + k0;
                    const int yy = zero ? y : ext_coord(y, im.H, a.bmode);
                    const bool yok = idx < nchunks && (!zero || (y >= 0 && y < im.H));
                    const float *src = im.img + (int64_t)(yok ? yy : 0) * im.pitch;
                    if (zero && yok && k0 + 8 <= ncols && gx0 >= 0 && gx0 + 8 <= im.W &&
                        (reinterpret_cast<uintptr_t>(src + gx0) & 15) == 0) {
                        const float4 p = __ldg(reinterpret_cast<const float4 *>(src + gx0));
                        const float4 q = __ldg(reinterpret_cast<const float4 *>(src + gx0 + 4));
                        v[uu][0] = p.x; v[uu][1] = p.y; v[uu][2] = p.z; v[uu][3] = p.w;
                        v[uu][4] = q.x; v[uu][5] = q.y; v[uu][6] = q.z; v[uu][7] = q.w;
                    } else {
#pragma unroll
                        for (int t = 0; t < 8; ++t) {
                            const int k = k0 + t, gx = gx0 + t;
                            const int xx = zero ? ((gx >= 0 && gx < im.W) ? gx : -1) : ext_coord(gx, im.W, a.bmode);
                            v[uu][t] = (yok && k < ncols && xx >= 0) ? __ldg(src + xx) : cen;   // cen: 0 after - cen
                        }
                    }
                }
#pragma unroll
                for (int uu = 0; uu < kU; ++uu) {
                    const int idx = base + uu * NP;
                    if (idx >= nchunks) break;
                    const int r = idx / nk8, k0 = 8 * (idx - r * nk8);
#pragma unroll
                    for (int t = 0; t < 8; ++t) v[uu][t] = (v[uu][t] - cen) * sc;
                    if constexpr (SPLIT) {   // BF16 hi + lo
                        uint32_t hw[4], lw[4];
#pragma unroll
                        for (int t = 0; t < 4; ++t) b2split(v[uu][2 * t], v[uu][2 * t + 1], hw[t], lw[t]);
                        *reinterpret_cast<uint4 *>(dP + sw128_offset(TY, r, k0)) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
                        *reinterpret_cast<uint4 *>(dP + plo + sw128_offset(TY, r, k0)) =
                            make_uint4(lw[0], lw[1], lw[2], lw[3]);
                    } else {
                        *reinterpret_cast<uint4 *>(dP + sw128_offset(TY, r, k0)) =
                            make_uint4(h2pack(v[uu][0], v[uu][1]), h2pack(v[uu][2], v[uu][3]),
                                       h2pack(v[uu][4], v[uu][5]), h2pack(v[uu][6], v[uu][7]));
                    }
                }
            }
            fence_proxy_async_smem();
            named_barrier(1, NP);   // P built
            if (ptid == 0) mbar_arrive(&p_full[pb]);
        }
    } else {
        // -------------------------------------------------------------- epilogue
        // TMEM lane n = 2 x' + part, x' = 63 - x (the operand strip runs backwards in x): warp w
        // reads quarter w & 3 (x' 16 (w & 3) .. + 15) and rows [rbase, rbase + TY / 2), and
        // stores its part of J (signal 2 unit + part of the intermediate; the column pass
        // demodulates nothing, its taps are modulated too).
        const int quarter = warp & 3, half = warp >> 2;
        const uint32_t lane_base = (uint32_t)(32 * quarter) << 16;
        const int rpw = TY / 2, rbase = half * rpw;
        const int part = lane & 1, xl = kMtTileX - 1 - (16 * quarter + (lane >> 1));
        int job = 0;
        for (int it = blockIdx.x; it < nitems && !*abort_s; it += gridDim.x) {
            const RowItem w = row_item_mt(a, D, it);
            const int y0 = w.y0;
            const TcImgView im = tc_img(a, w.img);
            float cen_unused;
            int e;
            tc_centre(a, w.img, cen_unused, e);
            const TcFreqDev f = D.freqs[w.s];
            const float unscale = ldexpf(f.unscale_row, e);
            const int gx = w.x0 + xl;
            const bool xin = gx < im.W;
            const int u0 = f.u0, nu = a.nu_f;
            bool ok = true;
            for (int q = 0; q < nu; ++q, ++job) {
                const int b = job & 1;
                if (!mbar_wait(&tmem_full[b], (job >> 1) & 1, abort_s)) {
                    ok = false;
                    break;
                }
                // job's MMAs are complete: its Am buffer takes the copy of job + kAmBufs
                if (warp == 0 && lane == 0 && job + kAmBufs < njobs_row) {
                    issue_am(job + kAmBufs);
                    *issued_s = job + kAmBufs + 1;
                }
                __syncwarp();
                tc_fence_after();
                const int64_t pstride = (int64_t)im.Wq * 2 * im.Hp;   // between planes
                const int64_t bstride = (int64_t)im.Wq * 16;          // between 8-row blocks
                // the unit's plane (and the next one, lo, under split); Re J, Im J interleaved
                uint16_t *dst0 = im.sig + (int64_t)np * (u0 + q) * pstride + (int64_t)((a.Lpad + y0) >> 3) * bstride +
                                 (int64_t)(xin ? gx : 0) * 16 + part * 8;
#pragma unroll 1
                for (int c0 = rbase; c0 < rbase + rpw; c0 += 16) {
                    float v[16];
                    tmem_ld16(tmem + lane_base + (uint32_t)TY * b + c0, v);
                    uint32_t pk[2][4], pl[2][4];   // [8-row block][row pair]
                    if constexpr (SPLIT) {
#pragma unroll
                        for (int j = 0; j < 16; j += 2)
                            b2split(v[j] * unscale, v[j + 1] * unscale, pk[j >> 3][(j & 7) >> 1], pl[j >> 3][(j & 7) >> 1]);
                    } else {
#pragma unroll
                        for (int j = 0; j < 16; j += 2) pk[j >> 3][(j & 7) >> 1] = h2pack(v[j] * unscale, v[j + 1] * unscale);
                    }
                    if (xin) {
#pragma unroll
                        for (int blk = 0; blk < 2; ++blk) {
                            const int64_t o = (int64_t)((c0 + 8 * blk) >> 3) * bstride;
                            *reinterpret_cast<uint4 *>(dst0 + o) = make_uint4(pk[blk][0], pk[blk][1], pk[blk][2], pk[blk][3]);
                            if constexpr (SPLIT)
                                *reinterpret_cast<uint4 *>(dst0 + pstride + o) =
                                    make_uint4(pl[blk][0], pl[blk][1], pl[blk][2], pl[blk][3]);
                        }
                    }
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(&tmem_empty[b]);
            }
            if (!ok) {
                if (lane == 0) fail_status(a.status, abort_s, 28);
                break;
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 15 && lane == 0) {
        // Am copies issued but not waited for (after a stop) land before shared memory is
        // released; copy i went to buffer i % kAmBufs as its (i / kAmBufs)-th use
        const int issued = max(*issued_s, min(kAmBufs, njobs_row));
        for (int i = *landed_s; i < issued; ++i) {
            volatile int dummy = 0;
            mbar_wait(&a_full[i % kAmBufs], (i / kAmBufs) & 1, &dummy);
        }
    }
    if (a.p_tma && warp == kMtEpiWarps && lane == 0) {
        // the same for the P loads: item i's went to buffer i & 1 as its (i / 2)-th use
        for (int i = *p_landed_s; i < *p_issued_s; ++i) {
            volatile int dummy = 0;
            mbar_wait(&p_full[i & 1], (i >> 1) & 1, &dummy);
        }
    }
    if (warp == 0) tmem_dealloc(tmem, 128);
}

// Strip of a modulated Toeplitz operand (see tstrip_cores): core j, row r, element c holds
// S(d) (cos, -sin)(w d) 2^sB for row part r & 1, d = 4 j + c + r / 2 - off, zero outside
// |d| <= R; FP64, rounded to FP16.  Row pass (Am): off = 63 + R8, w = w^c (rows x of the 64-
// column tile backwards, k the input column from x0 - R8 on).  Column pass (Gm): off =
// TYC - 1 + R8, w = w^s (rows y of the job backwards, l the window row from y0 - R8 on).
// split = 1: BF16 instead, hi = bf16(v) in Q[0 .. n) and lo = bf16(v - hi) in Q[n .. 2 n).
__global__ void k_build_tstrip(uint16_t *__restrict__ Q, int ncores, int off, int R, double sigma, double w, int sB,
                               int split)
{
    const int n = 64 * ncores;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int j = i >> 6, r = (i >> 3) & 7, c = i & 7;
        const int d = 4 * j + c + (r >> 1) - off;
        double v = 0.0;
        if (d >= -R && d <= R) {
            const double g = exp(-(double)d * d / (2.0 * sigma * sigma)) / (2.5066282746310002 * sigma);
            v = ldexp((r & 1) ? -g * sin(w * d) : g * cos(w * d), sB);
        }
        if (split) {
            const __nv_bfloat16 hi = __float2bfloat16_rn((float)v);
            Q[i] = __bfloat16_as_ushort(hi);
            Q[n + i] = __bfloat16_as_ushort(__float2bfloat16_rn((float)(v - (double)__bfloat162float(hi))));
        } else {
            Q[i] = __half_as_ushort(__float2half_rn((float)v));
        }
    }
}

// --------------------------------------------------------- column pass, modulated taps
// With the modulated-tap row pass the intermediate holds J itself (Re J, Im J per unit) and
// the column pass of Eq. 7-9 is one product with a per-unit operand of modulated taps,
//   D[(x, re|im of J)][(y, re|im of G)] = sum_l J[(x, .)][l] Gm[(y, .)][l],
//   Gm[(y, re)][l] = S(d) cos(w^s d),  Gm[(y, im)][l] = -S(d) sin(w^s d),  d = l - y - R8,
// whose four real sums per (x, y) give F_theta = sum G J and F_{pi-theta} = sum G J*
// (Eq. 13-16) with two additions each: no row phases at all.  Operand rows n = 2 x + part,
// columns m = 2 y + part, so the sums of a column meet by one shuffle.  Items: (unit,
// 64-column tile, 64-row tile; 32-row tiles, MMA N = 64, when the two-deep operands of 64 rows
// exceed shared memory, as for radius 96).  One producer warp (lane 0) loads each job's J boxes
// by TMA and its unit's Gm by bulk copies, two jobs deep, and issues the MMAs into two TMEM
// accumulators; 16 epilogue warps (one row quarter x one TMEM lane quarter each) read their
// accumulator columns with one wait, release the accumulator, add the c A(x) B(y) correction
// and store complex64.
constexpr int kMtColAcc = 2;       // TMEM accumulators (128 columns each)
constexpr int kMtColEpiWarps = 16;
constexpr int kMtColMaxStages = 3;   // operand stages of the modulated-tap column kernel
constexpr int kMtColThreads = 32 * (kMtColEpiWarps + 2);   // + the MMA warp and the copy warp

struct MtColSmem {
    uint32_t a_off, b_off, c_off, desc_off, bar_off, misc_off, total;
};

// TYC: output rows per job (64; 32 when the operands of 64 do not fit); the B operand is the
// unit's strip of 2 TYC rows x K.  nst operand stages; split = 1: hi and lo of both operands.
__host__ __device__ inline MtColSmem mt_col_smem(int K, int TYC, int split = 0, int nst = 2)
{
    MtColSmem L;
    const uint32_t np = split ? 2u : 1u;
    L.a_off = 0;                                        // [nst][np] x 128 x K (no swizzle, core matrices)
    L.b_off = L.a_off + nst * np * 128u * K * 2;        // [nst][np] strips of 2 TYC rows x K
    L.c_off = L.b_off + nst * np * tstrip_bytes(K, 2 * TYC);   // [nst] correction operands A, B
    L.desc_off = (L.c_off + nst * 2u * kCorrBlockHalfs * 2 + 127) & ~127u;
    L.bar_off = L.desc_off + kDescBytes;
    L.misc_off = L.bar_off + 16 * 8;
    L.total = L.misc_off + 64;
    return L;
}

struct MtColItem {
    int unit, x0, y0;
    int img;     // image of a batch (0 for one image)
};
__device__ __forceinline__ MtColItem col_item_mt(const TcBankArgs &a, const TcDesc &d, int it)
{
    if (a.col_list) {
        const int4 v = a.col_list[it];
        return MtColItem{v.y, v.z, v.w, v.x};
    }
    const int g = it / a.col_cnt, local = it - g * a.col_cnt;
    const int per_unit = a.col_ny * a.col_nx64;
    const int q = local / per_unit, rest = local - q * per_unit;
    const TcFreqDev f = d.freqs[d.forder[g]];
    return MtColItem{f.u0 + q, (rest % a.col_nx64) * 64, (rest / a.col_nx64) * a.col_mt_ty, 0};
}

// SPLIT: BF16 operands as hi + lo pairs (a.split); a.col_mt_nst operand stages.
template <bool SPLIT>
__global__ void __launch_bounds__(kMtColThreads, 1) k_gabor_tc_cols_mt(const __grid_constant__ TcBankArgs a)
{
    const int nitems = a.col_list ? a.n_col : a.nf * a.col_cnt;
    extern __shared__ unsigned char smem_dyn[];
    unsigned char *sm = reinterpret_cast<unsigned char *>(((uintptr_t)smem_dyn + 1023) & ~(uintptr_t)1023);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int TYC = a.col_mt_ty;
    const int NST = a.col_mt_nst;
    constexpr int np = SPLIT ? 2 : 1;
    const MtColSmem L = mt_col_smem(a.col_kmax, TYC, SPLIT ? 1 : 0, NST);
    unsigned char *sA = sm + L.a_off;
    unsigned char *sB = sm + L.b_off;
    unsigned char *sC = sm + L.c_off;
    uint64_t *bars = reinterpret_cast<uint64_t *>(sm + L.bar_off);
    uint64_t *tmem_full = bars;            // [2] commit
    uint64_t *tmem_empty = bars + 2;       // [2] epilogue warps
    uint64_t *ab_full = bars + 4;          // [kMtColMaxStages] TMA + bulk-copy bytes of a job's operands
    uint64_t *ab_empty = bars + 4 + kMtColMaxStages;   // [kMtColMaxStages] commit: the MMA reading them is done
    uint64_t *drain = bars + 4 + 2 * kMtColMaxStages;
    uint32_t *tmem_s = reinterpret_cast<uint32_t *>(sm + L.misc_off);
    volatile int *abort_s = reinterpret_cast<volatile int *>(sm + L.misc_off + 4);
    volatile int *issued_s = reinterpret_cast<volatile int *>(sm + L.misc_off + 8);   // jobs whose copies were issued
    volatile int *landed_s = reinterpret_cast<volatile int *>(sm + L.misc_off + 12);  // jobs whose copies were waited for
    volatile int *stage_k = reinterpret_cast<volatile int *>(sm + L.misc_off + 16);   // [kMtColMaxStages] K of the staged job
    const uint32_t ahalf = 128u * a.col_kmax * 2;                 // one A operand (hi, or lo under split)
    const uint32_t obuf = np * ahalf;                             // the A operands of a stage
    const uint32_t gbuf = np * tstrip_bytes(a.col_kmax, 2 * TYC); // the B strips of a stage
    const TcDesc D = load_desc(a, sm + L.desc_off);

    if (tid == 0) {
        for (int i = 0; i < 2; ++i) {
            mbar_init(&tmem_full[i], 1);
            mbar_init(&tmem_empty[i], kMtColEpiWarps);
        }
        for (int i = 0; i < kMtColMaxStages; ++i) {
            mbar_init(&ab_full[i], 1);
            mbar_init(&ab_empty[i], 1);
        }
        mbar_init(drain, 1);
        *abort_s = 0;
        *issued_s = 0;
        *landed_s = 0;
        mbar_fence_init();
    }
    if (warp == 0) {
        tmem_alloc(tmem_s, 128 * kMtColAcc);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    // programmatic dependent of the row pass: the set-up above overlaps its tail; J, the F[1]
    // tables and the centre are read after it completed
    pdl_wait();
    const uint32_t tmem = *tmem_s;
    const uint32_t idesc = idesc_f16(SPLIT ? 1 : 0, 128, 2 * TYC);
    const int njobs = nitems > (int)blockIdx.x ? (nitems - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;

    auto item = [&](int j) { return col_item_mt(a, D, blockIdx.x + j * gridDim.x); };
    if (warp == kMtColEpiWarps + 1) {
        // -------------------------------------------------------------- copies (lane 0)
        // job j's operands into stage j % NST once the MMAs of job j - NST are done with it: J
        // boxes (64 columns x both parts x 8 rows of a block x 8 blocks of the unit's plane,
        // landing as K-major core matrices with operand row n = 2 x + part; under split the hi
        // plane, then the lo plane), the unit's Gm strips (one bulk copy: hi, then lo under
        // split) and the correction operands.  A warp of its own, so that issuing the copies
        // overlaps the MMA warp's issue of the previous job's products.
        if (lane == 0) {
            if (a.imgs == nullptr) prefetch_tmap(&a.tmA[0]);
            int j = 0;
            for (; j < njobs; ++j) {
                if (*abort_s) break;
                const int st = j % NST;
                if (j >= NST && !mbar_wait(&ab_empty[st], ((j - NST) / NST) & 1, abort_s)) {
                    fail_status(a.status, abort_s, 38);
                    break;
                }
                const MtColItem w = item(j);
                const TcUnitDev u = D.units[w.unit];
                const TcFreqDev f = D.freqs[u.s];
                const int nkb = f.Kcol / 64;
                const uint32_t bbytes = tstrip_bytes(f.Kcol, 2 * TYC);
                stage_k[st] = f.Kcol;   // read by the MMA thread after the stage's barrier completes
                mbar_arrive_expect_tx(&ab_full[st], np * (nkb * 16384u + bbytes) + 4u * kCorrBlockHalfs);
                const int yb0 = (a.Lpad + w.y0 - f.R8) >> 3;
                const uint32_t dst = smem_u32(sA + st * obuf);
                const TcImgView im = tc_img(a, w.img);
                // boxes of 16 columns x both parts x 8 rows (512 contiguous bytes) x 4 x 8 blocks
                const int pb = (int)(im.Hp >> 3);
                for (int h = 0; h < np; ++h)
                    for (int kb = 0; kb < nkb; ++kb)
                        tma_load_3d(dst + h * ahalf + kb * 16384u, im.tm, 0, w.x0 / 16,
                                    (np * w.unit + h) * pb + yb0 + 8 * kb, &ab_full[st]);
                bulk_load(smem_u32(sB + st * gbuf), u.Gm, np * bbytes, &ab_full[st]);
                // the correction operands of (unit, x0) and (unit, y0)
                const int nxb = (im.W + 63) / 64, nyb = (im.H + TYC - 1) / TYC;
                const uint32_t cdst = smem_u32(sC + st * 4u * kCorrBlockHalfs);
                bulk_load(cdst, im.corrA + ((int64_t)w.unit * nxb + w.x0 / 64) * kCorrBlockHalfs, 2u * kCorrBlockHalfs,
                          &ab_full[st]);
                bulk_load(cdst + 2u * kCorrBlockHalfs, im.corrB + ((int64_t)w.unit * nyb + w.y0 / TYC) * kCorrBlockHalfs,
                          2u * kCorrBlockHalfs, &ab_full[st]);
            }
            *issued_s = j;
        }
    } else if (warp == kMtColEpiWarps) {
        // -------------------------------------------------------------- MMAs (lane 0)
        if (lane == 0) {
            int landed = 0;
            for (int j = 0; j < njobs; ++j) {
                if (*abort_s) break;
                const int st = j % NST, acc = j & 1;
                if (!mbar_wait(&ab_full[st], (j / NST) & 1, abort_s)) {
                    fail_status(a.status, abort_s, 36);
                    break;
                }
                const int Kcol = stage_k[st];
                landed = j + 1;
                if (j >= kMtColAcc && !mbar_wait(&tmem_empty[acc], ((j - kMtColAcc) >> 1) & 1, abort_s)) {
                    fail_status(a.status, abort_s, 37);
                    break;
                }
                tc_fence_after();
                const uint32_t a0 = smem_u32(sA + st * obuf), b0 = smem_u32(sB + st * gbuf);
                const uint32_t a0l = a0 + ahalf, b0l = b0 + tstrip_bytes(Kcol, 2 * TYC);
                for (int kb = 0; kb < Kcol / 64; ++kb)
#pragma unroll
                    for (int kk = 0; kk < 4; ++kk) {
                        const uint32_t ao = kb * 16384 + kk * 4096;
                        tc_mma_f16(tmem + 128u * acc, smem_desc_kmajor(a0 + ao, 2048, 128), tstrip_desc(b0, 4 * kb + kk),
                                   idesc, (kb | kk) != 0);
                        if constexpr (SPLIT) {   // J_hi G_lo + J_lo G_hi (the lo x lo product is dropped)
                            tc_mma_f16(tmem + 128u * acc, smem_desc_kmajor(a0 + ao, 2048, 128),
                                       tstrip_desc(b0l, 4 * kb + kk), idesc, 1);
                            tc_mma_f16(tmem + 128u * acc, smem_desc_kmajor(a0l + ao, 2048, 128),
                                       tstrip_desc(b0, 4 * kb + kk), idesc, 1);
                        }
                    }
                // + c A(x) B(y), the bank's response to the constant image c: one K = 16 product
                {
                    const uint32_t c0 = smem_u32(sC + st * 4u * kCorrBlockHalfs);
                    tc_mma_f16(tmem + 128u * acc, smem_desc_kmajor(c0, 2048, 128),
                               smem_desc_kmajor(c0 + 2u * kCorrBlockHalfs, 2048, 128), idesc, 1);
                }
                tc_commit(&tmem_full[acc]);
                tc_commit(&ab_empty[st]);
            }
            *landed_s = landed;
            tc_commit(drain);
            if (!mbar_wait(drain, 0, abort_s)) {
                volatile int dummy = 0;
                mbar_wait(drain, 0, &dummy);
            }
        }
    } else {
        // -------------------------------------------------------------- epilogue
        // TMEM lane n = 2 x + part (part 0: Re J, 1: Im J), column m = 2 y' + g (g 0: Re G,
        // 1: Im G), y' = TYC - 1 - y (the Gm strip runs backwards in y).  Warp w reads lane
        // quarter w & 3 (columns x 16 (w & 3) .. + 15) and the TYC / 4 rows y from (TYC / 4) (w >> 2)
        // on, one block of 2 TYC / 4 accumulator columns, with one or two 16-column loads waited
        // for once.  The part-0 lane of a column stores F_theta, the part-1 lane F_{pi - theta}
        // (paired units).
        const int quarter = warp & 3, rq = warp >> 2;
        const int rpw = TYC / 4;                       // rows per warp: 16 or 8
        const uint32_t lane_base = (uint32_t)(32 * quarter) << 16;
        const int part = lane & 1, xl = 16 * quarter + (lane >> 1);
        for (int j = 0; j < njobs; ++j) {
            const MtColItem w = col_item_mt(a, D, blockIdx.x + j * gridDim.x);
            const TcImgView im = tc_img(a, w.img);
            const TcUnitDev u = D.units[w.unit];
            const TcFreqDev f = D.freqs[u.s];
            const int acc = j & 1;
            const bool paired = u.plane_b >= 0;
            const int x = w.x0 + xl, ybase = w.y0 + rpw * rq;
            const bool xok = x < im.W;
            const int plane = part ? u.plane_b : u.plane_a;
            const bool store = xok && (part == 0 || paired);
            const int nrows = min(rpw, im.H - ybase);
            const int64_t ostep = a.layout ? (int64_t)im.W * a.nplanes : (int64_t)im.W;
            float2 *o = im.out + tc_out_offset(a, im, store ? plane : 0, max(ybase, 0), xok ? x : 0);
            if (!mbar_wait(&tmem_full[acc], (j >> 1) & 1, abort_s)) {
                if (lane == 0) fail_status(a.status, abort_s, 39);
                break;
            }
            tc_fence_after();
            uint32_t r[32];
            const uint32_t ta = tmem + lane_base + 128u * acc + 2 * (TYC - rpw * (rq + 1));
            tmem_ld16_async(ta, *reinterpret_cast<uint32_t(*)[16]>(&r[0]));
            if (rpw == 16) tmem_ld16_async(ta + 16, *reinterpret_cast<uint32_t(*)[16]>(&r[16]));
            tmem_wait_ld();
            // the accumulator is free for the next job's MMA once the values are in registers
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&tmem_empty[acc]);
            const float unscale = f.unscale_col;
            // loaded value pair tt belongs to row t = rpw - 1 - tt (the strip runs backwards in
            // y): walk the rows from the last one up, keeping the register index static
            o += (int64_t)(rpw - 1) * ostep;
#pragma unroll
            for (int tt = 0; tt < 16; ++tt) {
                if (tt >= rpw) break;
                const int t = rpw - 1 - tt;
                // this lane: (sum Re G, sum Im G) x (its part of J); the partner lane the other part
                const float gr = __uint_as_float(r[2 * tt]) * unscale, gi = __uint_as_float(r[2 * tt + 1]) * unscale;
                const float or_ = __shfl_xor_sync(0xffffffffu, gr, 1), oi = __shfl_xor_sync(0xffffffffu, gi, 1);
                // part 0 (A = gr, C = gi, D = or_, B = oi): F_theta = (A - B, C + D);
                // part 1 (D = gr, B = gi, A = or_, C = oi): F_{pi-theta} = (A + B, C - D)
                // (the correction c A(x) B(y), c conj(A(x)) B(y) for pi - theta, is in the sums)
                const float fr = part ? or_ + gi : gr - oi;
                const float fi = part ? oi - gr : gi + or_;
                if (store && t < nrows) __stcs(o, make_float2(fr, fi));
                o -= ostep;
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == kMtColEpiWarps && lane == 0) {
        // copies issued but not waited for (after a stop) land before shared memory is released;
        // at most one per stage is outstanding
        for (int jj = *landed_s; jj < *issued_s; ++jj) {
            volatile int dummy = 0;
            mbar_wait(&ab_full[jj % NST], (jj / NST) & 1, &dummy);
        }
    }
    if (warp == 0) tmem_dealloc(tmem, 128 * kMtColAcc);
}

// --------------------------------------------------------------------------- column pass
// Items: (unit, x0, y0), sorted by frequency; paired units take 32 columns x 4 signals,
// unpaired ones 64 columns x 2 signals (always 128 A rows).  One producer warp keeps NST - 1
// jobs of A-operand TMA loads in flight ahead of the MMA (NST A buffers).  A box of 8 rows of
// a block x 32 (64) columns x 4 (2) signals x 8 row blocks of the blocked intermediate lands
// as 8 x 8-element core matrices: operand row n = 32 s + x (64 s + x), element (n, k) at
// (k / 8) * 2048 + n * 16 + (k % 8) * 2 bytes, the MMA's K-major layout without swizzle (core
// matrices 128 bytes apart along n, 2048 along k).  Epilogue: every warp moves its TMEM lane
// quarter (one signal for 32 columns) to shared memory and releases the accumulator; then
// each warp remodulates 8 of the 64 rows for every column of the tile.  Epilogue: every warp moves
// its TMEM lane quarter (one signal for 32 columns) to shared memory and releases the
// accumulator; then each warp remodulates 16 of the 64 rows for every column of the tile.
constexpr int kColEpiWarps = 8;                           // warps 0-7; warp 8 produces
constexpr int kColThreads = 32 * (kColEpiWarps + 1);

__global__ void __launch_bounds__(kColThreads, 1) k_gabor_tc_cols(const __grid_constant__ TcBankArgs a)
{
    const int nitems = a.nf * a.col_cnt;
    extern __shared__ unsigned char smem_dyn[];
    unsigned char *sm = reinterpret_cast<unsigned char *>(((uintptr_t)smem_dyn + 1023) & ~(uintptr_t)1023);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int NST = a.col_nst;
    const ColSmem L = col_smem(a.col_kmax, NST);
    unsigned char *sG = sm + L.g_off;
    unsigned char *sA = sm + L.a_off;                 // [NST] buffers of 128 x Kmax
    float *xch = reinterpret_cast<float *>(sm + L.xch_off);   // [4 quarters][64 rows][32 lanes]
    uint64_t *bars = reinterpret_cast<uint64_t *>(sm + L.bar_off);
    uint64_t *tmem_full = bars;                  // [kColAcc] commit
    uint64_t *tmem_empty = bars + kColAcc;       // [kColAcc] 8 epilogue warps
    uint64_t *a_empty = bars + 2 * kColAcc;      // [kColMaxStages] commit
    uint64_t *drain = bars + 2 * kColAcc + kColMaxStages;
    uint64_t *a_full = bars + 2 * kColAcc + kColMaxStages + 1;   // [kColMaxStages] TMA bytes
    uint64_t *g_full = bars + 2 * kColAcc + 2 * kColMaxStages + 1;   // G of a frequency landed
    uint32_t *tmem_s = reinterpret_cast<uint32_t *>(sm + L.misc_off);
    volatile int *abort_s = reinterpret_cast<volatile int *>(sm + L.misc_off + 4);
    const uint32_t abuf = 128u * a.col_kmax * 2;
    const TcDesc D = load_desc(a, sm + L.desc_off);
    float cen;
    int e_unused;
    image_centre(a, cen, e_unused);

    if (tid == 0) {
        for (int i = 0; i < kColAcc; ++i) {
            mbar_init(&tmem_full[i], 1);
            mbar_init(&tmem_empty[i], kColEpiWarps);
        }
        for (int i = 0; i < kColMaxStages; ++i) {
            mbar_init(&a_empty[i], 1);
            mbar_init(&a_full[i], 1);
        }
        mbar_init(g_full, 1);
        mbar_init(drain, 1);
        *abort_s = 0;
        mbar_fence_init();
    }
    if (warp == 0) {
        tmem_alloc(tmem_s, 64 * kColAcc);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_s;
    const uint32_t idesc = idesc_f16(0, 128, kColTileY);
    const int njobs = nitems > (int)blockIdx.x ? (nitems - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;

    if (warp == kColEpiWarps) {
        // -------------------------------------------------------------- producer warp
        // Lane 0 loads G (one bulk copy) when the frequency changes, keeps NST - 1 jobs of
        // A-operand TMA loads in flight ahead of the MMA, and issues the MMAs.
        auto item = [&](int j) { return col_item(a, D, blockIdx.x + j * gridDim.x); };
        int g_loads = 0, g_landed = 0;   // G copies issued / waited for (lane 0)
        // Job j's A operand into buffer j % NST: one box per 64 rows of the window (rows n of
        // the operand = signal n / xw, column x0 + n % xw; zeros beyond the image width).
        auto issue = [&](int j) {
            const ColItem w = item(j);
            const TcUnitDev u = D.units[w.unit];
            const TcFreqDev f = D.freqs[u.s];
            const int st = j % NST;
            const void *tm = u.plane_b >= 0 ? (const void *)&a.tmA[0] : (const void *)&a.tmA[1];
            mbar_arrive_expect_tx(&a_full[st], 128u * f.Kcol * 2);
            const int yb0 = (a.Lpad + w.y0 - f.R8) >> 3;   // first 8-row block of the window
            const uint32_t dst = smem_u32(sA + st * abuf);
            for (int kb = 0; kb < f.Kcol / 64; ++kb)
                tma_load_4d(dst + kb * 16384u, tm, 0, w.x0, (int)u.sig_idx, yb0 + 8 * kb, &a_full[st]);
        };
        int issued = 0, landed = 0;   // jobs whose loads were issued / waited for (lane 0)
        if (lane == 0)
            for (; issued < NST - 1 && issued < njobs; ++issued) issue(issued);
        int cur_s = -1;
        bool ok = true;
        for (int j = 0; j < njobs && ok; ++j) {
            if (__shfl_sync(0xffffffffu, (int)*abort_s, 0)) break;
            // G of job j's frequency: every earlier MMA must be done with the previous G
            const int sj = D.units[item(j).unit].s;
            if (sj != cur_s) {
                bool failed = false;
                if (lane == 0) {
                    failed = j >= 1 && !mbar_wait(&a_empty[(j - 1) % NST], ((j - 1) / NST) & 1, abort_s);
                    if (!failed) {
                        const uint32_t gbytes = kColTileY * D.freqs[sj].Kcol * 2;
                        mbar_arrive_expect_tx(g_full, gbytes);
                        bulk_load(smem_u32(sG), D.freqs[sj].Bcol, gbytes, g_full);
                        ++g_loads;
                        failed = !mbar_wait(g_full, (g_loads - 1) & 1, abort_s);
                        if (!failed) g_landed = g_loads;
                    }
                }
                if (__shfl_sync(0xffffffffu, failed, 0)) {
                    if (lane == 0) fail_status(a.status, abort_s, 34);
                    break;
                }
                cur_s = sj;
            }
            if (lane == 0) {
                const int b = j % kColAcc, st = j % NST;
                const TcFreqDev f = D.freqs[sj];
                const bool got = mbar_wait(&a_full[st], (j / NST) & 1, abort_s);
                if (got) landed = j + 1;
                if (!got) {
                    fail_status(a.status, abort_s, 35);
                    ok = false;
                } else if (j >= kColAcc && !mbar_wait(&tmem_empty[b], ((j - kColAcc) / kColAcc) & 1, abort_s)) {
                    fail_status(a.status, abort_s, 32);
                    ok = false;
                } else {
                    tc_fence_after();
                    const uint32_t a0 = smem_u32(sA + st * abuf), g0 = smem_u32(sG);
                    for (int kb = 0; kb < f.Kcol / 64; ++kb)
#pragma unroll
                        for (int kk = 0; kk < 4; ++kk)
                            tc_mma_f16(tmem + 64u * b, smem_desc_kmajor(a0 + kb * 16384 + kk * 4096, 2048, 128),
                                       smem_desc_sw128(g0 + kb * kColTileY * 128) + 2 * kk, idesc, (kb | kk) != 0);
                    tc_commit(&tmem_full[b]);
                    tc_commit(&a_empty[st]);
                    // refill: job j + NST - 1 goes into the buffer that job j - 1's MMA read
                    const int jn = j + NST - 1;
                    if (jn < njobs) {
                        if (j >= 1 && !mbar_wait(&a_empty[(j - 1) % NST], ((j - 1) / NST) & 1, abort_s)) {
                            fail_status(a.status, abort_s, 31);
                            ok = false;
                        } else {
                            issue(jn);
                            issued = jn + 1;
                        }
                    }
                }
            }
            ok = __shfl_sync(0xffffffffu, ok, 0);
        }
        if (lane == 0) {
            // drain: every MMA is complete, and every TMA load issued has landed, before TMEM
            // and shared memory are released
            tc_commit(drain);
            if (!mbar_wait(drain, 0, abort_s)) {
                volatile int dummy = 0;
                mbar_wait(drain, 0, &dummy);
            }
            // loads issued but not waited for (after an abort) land before shared memory is
            // released
            for (int jj = landed; jj < issued; ++jj) {
                volatile int dummy = 0;
                mbar_wait(&a_full[jj % NST], (jj / NST) & 1, &dummy);
            }
            if (g_landed < g_loads) {
                volatile int dummy = 0;
                mbar_wait(g_full, (g_loads - 1) & 1, &dummy);
            }
        }
    } else {
        // -------------------------------------------------------------- epilogue
        // D[n][y]: lane quarter q holds rows 32q .. 32q+31 of n.
        //   paired:   quarter 0 P, 1 Q (theta), 2 P', 3 Q' (pi - theta), x = lane
        //   unpaired: quarters 0-1 P (x = 32 q + lane), quarters 2-3 Q
        // Warps w and w + 4 read quarter w & 3 (columns y split in halves); then warp w
        // remodulates rows 8w .. 8w+7 of the tile.
        const int quarter = warp & 3, half = warp >> 2;
        const uint32_t lane_base = (uint32_t)(32 * quarter) << 16;
        for (int j = 0; j < njobs; ++j) {
            const ColItem w = col_item(a, D, blockIdx.x + j * gridDim.x);
            const TcUnitDev u = D.units[w.unit];
            const TcFreqDev f = D.freqs[u.s];
            const int x0 = w.x0, y0 = w.y0, b = j % kColAcc;
            const bool paired = u.plane_b >= 0;
            // row phases: lane l holds row y0 + 8 warp + (l & 7)
            const int yr = y0 + 8 * warp + (lane & 7);
            const float2 pyr = yr < a.H ? __ldg(&u.phy[yr]) : make_float2(0.f, 0.f);
            // c B(y) for the same rows; A(x) for the lane's columns (the F[1] correction)
            const float2 byr = yr < a.H ? __ldg(&a.onesB[(int64_t)w.unit * a.H + yr]) : make_float2(0.f, 0.f);
            const int xa0 = x0 + lane, xa1 = x0 + 32 + lane;
            const float2 ax0 = xa0 < a.W ? __ldg(&a.onesA[(int64_t)w.unit * a.W + xa0]) : make_float2(0.f, 0.f);
            const float2 ax1 = (!paired && xa1 < a.W) ? __ldg(&a.onesA[(int64_t)w.unit * a.W + xa1]) : make_float2(0.f, 0.f);
            const bool failed = !mbar_wait(&tmem_full[b], (j / kColAcc) & 1, abort_s);
            if (named_barrier_or(2, 256, failed)) {
                if (tid == 0) fail_status(a.status, abort_s, 33);
                break;
            }
            tc_fence_after();
            const float unscale = f.unscale_col;
            const uint32_t tb = tmem + lane_base + 64u * b;
            float *xq = xch + quarter * (kColTileY * 32) + lane;
#pragma unroll 1
            for (int c0 = half * (kColTileY / 2); c0 < (half + 1) * (kColTileY / 2); c0 += 16) {
                float v[16];
                tmem_ld16(tb + c0, v);
#pragma unroll
                for (int jj = 0; jj < 16; ++jj) xq[(c0 + jj) * 32] = v[jj] * unscale;
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&tmem_empty[b]);   // the accumulator is free again
            named_barrier(2, 256);
            const float *xr = xch + (8 * warp) * 32 + lane;
#pragma unroll 4
            for (int r = 0; r < 8; ++r) {
                const int yy = y0 + 8 * warp + r;
                const float tx = __shfl_sync(0xffffffffu, pyr.x, r);
                const float ty = __shfl_sync(0xffffffffu, pyr.y, r);
                const float cbr = cen * __shfl_sync(0xffffffffu, byr.x, r);   // c B(y)
                const float cbi = cen * __shfl_sync(0xffffffffu, byr.y, r);
                if (yy < a.H) {
                    if (paired) {
                        const int x = x0 + lane;
                        if (x < a.W) {
                            const float P = xr[r * 32], Q = xr[(kColTileY + r) * 32];
                            const float P2 = xr[(2 * kColTileY + r) * 32], Q2 = xr[(3 * kColTileY + r) * 32];
                            // Eq. 7-8 (theta) and Eq. 15-16 (pi - theta), plus c A(x) B(y) and
                            // c conj(A(x)) B(y) (the response to c moves w^c to -w^c)
                            __stcs(a.out + tc_out_offset(a, u.plane_a, yy, x),
                                   make_float2(fmaf(tx, P, ty * Q) + (ax0.x * cbr - ax0.y * cbi),
                                               fmaf(ty, P, -tx * Q) + (ax0.x * cbi + ax0.y * cbr)));
                            __stcs(a.out + tc_out_offset(a, u.plane_b, yy, x),
                                   make_float2(fmaf(tx, P2, ty * Q2) + (ax0.x * cbr + ax0.y * cbi),
                                               fmaf(ty, P2, -tx * Q2) + (ax0.x * cbi - ax0.y * cbr)));
                        }
                    } else {
#pragma unroll
                        for (int h = 0; h < 2; ++h) {
                            const int x = x0 + 32 * h + lane;
                            const float2 ax = h ? ax1 : ax0;
                            if (x < a.W) {
                                const float P = xr[(h * kColTileY + r) * 32], Q = xr[((2 + h) * kColTileY + r) * 32];
                                __stcs(a.out + tc_out_offset(a, u.plane_a, yy, x),
                                       make_float2(fmaf(tx, P, ty * Q) + (ax.x * cbr - ax.y * cbi),
                                                   fmaf(ty, P, -tx * Q) + (ax.x * cbi + ax.y * cbr)));
                            }
                        }
                    }
                }
            }
            named_barrier(2, 256);   // xch is free for the next job
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0) tmem_dealloc(tmem, 64 * kColAcc);
}

// Min and max of the image as order-preserving keys, out[0] = ~min key and out[1] = max key
// (both words start at zero; one atomicMax pair per block).
__global__ void k_minmax(const float *__restrict__ img, int64_t pitch, int H, int W, unsigned *__restrict__ out)
{
    pdl_launch_dependents();   // k_ones may run alongside (it waits for this grid before it ends)
    unsigned lo = 0xffffffffu, hi = 0u;
    const int64_t ystep = (int64_t)gridDim.y * pitch;
    for (int x = blockIdx.x * blockDim.x + threadIdx.x; x < W; x += gridDim.x * blockDim.x) {
        int y = blockIdx.y;
        // four rows' loads in flight per thread
        for (; y + 3 * (int)gridDim.y < H; y += 4 * (int)gridDim.y) {
            const float *p = img + (int64_t)y * pitch + x;
            const unsigned k0 = fkey(__ldg(p)), k1 = fkey(__ldg(p + ystep)), k2 = fkey(__ldg(p + 2 * ystep)),
                           k3 = fkey(__ldg(p + 3 * ystep));
            lo = min(lo, min(min(k0, k1), min(k2, k3)));
            hi = max(hi, max(max(k0, k1), max(k2, k3)));
        }
        for (; y < H; y += gridDim.y) {
            const unsigned k = fkey(__ldg(img + (int64_t)y * pitch + x));
            lo = min(lo, k);
            hi = max(hi, k);
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        lo = min(lo, __shfl_xor_sync(0xffffffffu, lo, o));
        hi = max(hi, __shfl_xor_sync(0xffffffffu, hi, o));
    }
    __shared__ unsigned wlo[32], whi[32];
    if ((threadIdx.x & 31) == 0) {
        wlo[threadIdx.x >> 5] = lo;
        whi[threadIdx.x >> 5] = hi;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int i = 1; i < (int)(blockDim.x >> 5); ++i) {
            lo = min(lo, wlo[i]);
            hi = max(hi, whi[i]);
        }
        atomicMax(out, ~lo);
        atomicMax(out + 1, hi);
    }
}

// Batch form of k_minmax: grid (8, 8, images); block (bx, by) of image z writes the (~min, max)
// keys of its share of the image to partial bx + 8 by (kMmParts per image, no atomics and no
// zeroing; k_ones reduces them).
__global__ void k_minmax_batch(const TcBankArgs a)
{
    pdl_launch_dependents();
    const TcImgDev im = a.imgs[blockIdx.z];
    unsigned lo = 0xffffffffu, hi = 0u;
    for (int y = blockIdx.y; y < im.H; y += gridDim.y) {
        const float *row = im.img + (int64_t)y * im.pitch;
        for (int x = blockIdx.x * blockDim.x + threadIdx.x; x < im.W; x += gridDim.x * blockDim.x) {
            const unsigned k = fkey(__ldg(row + x));
            lo = min(lo, k);
            hi = max(hi, k);
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        lo = min(lo, __shfl_xor_sync(0xffffffffu, lo, o));
        hi = max(hi, __shfl_xor_sync(0xffffffffu, hi, o));
    }
    __shared__ unsigned wlo[32], whi[32];
    if ((threadIdx.x & 31) == 0) {
        wlo[threadIdx.x >> 5] = lo;
        whi[threadIdx.x >> 5] = hi;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int i = 1; i < (int)(blockDim.x >> 5); ++i) {
            lo = min(lo, wlo[i]);
            hi = max(hi, whi[i]);
        }
        unsigned *p = a.mm_part + ((int64_t)blockIdx.z * kMmParts + blockIdx.y * gridDim.x + blockIdx.x) * 2;
        p[0] = ~lo;
        p[1] = hi;
    }
}

// pre[u][0][j] = sum_{d=-R}^{-R+j-1} S(d) exp(i w^c d), pre[u][1][j] the same with w^s,
// j = 0 .. 2R+1 (FP64, phases reduced exactly: w d = pi (w / pi) d mod 2 pi).  One thread per
// (unit, direction).
__global__ void k_build_prefix(const double *__restrict__ unit_w, const TcUnitDev *__restrict__ units,
                               const TcFreqDev *__restrict__ freqs, const double *__restrict__ sigma, int nunits,
                               int stride, double2 *__restrict__ pre)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= 2 * nunits) return;
    const int u = i >> 1, dir = i & 1;
    const int s = units[u].s, R = freqs[s].R;
    const double sg = sigma[s], w = unit_w[2 * u + dir];
    double2 *p = pre + ((int64_t)u * 2 + dir) * stride;
    double re = 0.0, im = 0.0;
    p[0] = make_double2(0.0, 0.0);
    for (int d = -R; d <= R; ++d) {
        double sn, cs;
        sincospi(fmod(w * d, 2.0), &sn, &cs);
        const double g = exp(-(double)d * d / (2.0 * sg * sg)) / (2.5066282746310002 * sg);
        re += g * cs;
        im += g * sn;
        p[d + R + 1] = make_double2(re, im);
    }
}

// A[u][x] = sum over the in-image (zero rule) or all (other rules) taps d of S(d) exp(i w^c d),
// B[u][y] likewise along y: F[1](x, y) = A(x) B(y) for the unit's orientation.
// One entry of F[1] = A(x) B(y) (is_x: A at x = pos, else B at y = pos), from the unit's FP64
// prefix sums: the taps d with pos - d inside the image under the zero rule, all of them else.
__device__ __forceinline__ double2 ones_entry(const TcBankArgs &a, int R, int u, bool is_x, int pos, int n1)
{
    const double2 *pr = a.ones_pre + ((int64_t)u * 2 + (is_x ? 0 : 1)) * a.ones_stride;
    int lo = -R, hi = R;
    if (a.bmode == kBoundaryZero) {
        lo = max(-R, pos - (n1 - 1));
        hi = min(R, pos);
    }
    return make_double2(pr[hi + R + 1].x - pr[lo + R].x, pr[hi + R + 1].y - pr[lo + R].y);
}

// The correction operands of one image (layout in TcBankArgs): rows of 16 K elements, one per
// thread of the grid-stride loop.  A row of c A(x) 2^(sB - t) (Re or Im) and a row of B(y) 2^t
// hold parts whose products the MMA sums to a b within about 2^-22 |a b|: FP16 (a0, a0, a1)
// against (b0, b1, b0) with a = a0 + a1; BF16 (a0, a0, a1, a0, a1, a2) against
// (b0, b1, b0, b2, b1, b0) with a = a0 + a1 + a2.  2^t keeps |a| below 2^14 (|A|, |B| <= 1), so
// FP16 parts stay in range for |c| 2^sB < 2^29 (status code 60 beyond).
__device__ void corr_rows(const TcBankArgs &a, const TcUnitDev *__restrict__ units, const TcFreqDev *__restrict__ freqs,
                          int nunits, int W, int H, float c, uint16_t *cA, uint16_t *cB, int64_t gtid, int64_t gstride)
{
    const int TYC = a.col_mt_ty, nxb = (W + 63) / 64, nyb = (H + TYC - 1) / TYC;
    const int64_t nA = (int64_t)nunits * nxb * 128, n = nA + (int64_t)nunits * nyb * 128;
    for (int64_t i = gtid; i < n; i += gstride) {
        const bool isA = i < nA;
        const int64_t jj = isA ? i : i - nA;
        const int nb = isA ? nxb : nyb;
        const int u = (int)(jj / ((int64_t)nb * 128)), blk = (int)(jj / 128 % nb), row = (int)(jj % 128);
        const TcFreqDev f = freqs[units[u].s];
        const float inv = 1.f / f.unscale_col;   // 2^sB, exact
        const float amax = fabsf(c) * inv;        // bound of |c A(x)| 2^sB
        int t = 0;
        if (amax > 16384.f) frexpf(amax * (1.f / 16384.f), &t);
        if (t > 15) {
            if (!a.split && row == 0 && blk == 0) atomicExch(a.status, 60);
            t = 15;
        }
        float v = 0.f;
        if (isA) {
            const int x = 64 * blk + row / 2;
            if (x < W) {
                const double2 e = ones_entry(a, f.R, u, true, x, W);
                v = (float)(row & 1 ? e.y : e.x) * (c * inv) * ldexpf(1.f, -t);
            }
        } else {
            const int yp = row / 2, y = blk * TYC + TYC - 1 - yp;
            if (yp < TYC && y < H) {
                const double2 e = ones_entry(a, f.R, u, false, y, H);
                v = (float)(row & 1 ? e.y : e.x) * ldexpf(1.f, t);
            }
        }
        // parts: the residuals are exact in FP32
        uint16_t k[16] = {};
        if (a.split) {
            const __nv_bfloat16 p0 = __float2bfloat16_rn(v);
            const float r1 = v - __bfloat162float(p0);
            const __nv_bfloat16 p1 = __float2bfloat16_rn(r1);
            const __nv_bfloat16 p2 = __float2bfloat16_rn(r1 - __bfloat162float(p1));
            const __nv_bfloat16 sa[6] = {p0, p0, p1, p0, p1, p2}, sb[6] = {p0, p1, p0, p2, p1, p0};
            const __nv_bfloat16 *sl = isA ? sa : sb;
            for (int q = 0; q < 6; ++q) k[q] = *reinterpret_cast<const uint16_t *>(&sl[q]);
        } else {
            const __half p0 = __float2half_rn(v);
            const __half p1 = __float2half_rn(v - __half2float(p0));
            const __half sa[3] = {p0, p0, p1}, sb[3] = {p0, p1, p0};
            const __half *sl = isA ? sa : sb;
            for (int q = 0; q < 3; ++q) k[q] = *reinterpret_cast<const uint16_t *>(&sl[q]);
        }
        // element (row, k) at (k / 8) * 1024 + (row / 8) * 64 + (row % 8) * 8 + k % 8 halves
        uint16_t *base = (isA ? cA : cB) + ((int64_t)u * nb + blk) * kCorrBlockHalfs + (row / 8) * 64 + (row % 8) * 8;
        uint4 w0, w1;
        w0.x = k[0] | (uint32_t)k[1] << 16;
        w0.y = k[2] | (uint32_t)k[3] << 16;
        w0.z = k[4] | (uint32_t)k[5] << 16;
        w0.w = k[6] | (uint32_t)k[7] << 16;
        w1.x = k[8] | (uint32_t)k[9] << 16;
        w1.y = k[10] | (uint32_t)k[11] << 16;
        w1.z = k[12] | (uint32_t)k[13] << 16;
        w1.w = k[14] | (uint32_t)k[15] << 16;
        *reinterpret_cast<uint4 *>(base) = w0;
        *reinterpret_cast<uint4 *>(base + 1024) = w1;
    }
}

// The row pass's operand image (p_tma): P(x, y) = (f(x, y) - c) 2^-e as FP16, or as BF16 hi
// rows followed by H lo rows (split), pq elements per row; 8 columns per thread of the
// grid-stride loop (columns from W to the next multiple of 8 hold zeros).  The same arithmetic
// as the row kernel's producers, so both ways of building P give the same operand.
__device__ void operand_image(const float *__restrict__ img, int64_t pitch, int H, int W, float c, int e,
                              uint16_t *__restrict__ P, int64_t pq, int split, int64_t gtid, int64_t gstride)
{
    const float sc = ldexpf(1.f, -e);
    const int nx8 = (W + 7) / 8;
    const int64_t n = (int64_t)H * nx8;
    for (int64_t i = gtid; i < n; i += gstride) {
        const int y = (int)(i / nx8), x0 = 8 * (int)(i - (int64_t)y * nx8);
        const float *src = img + (int64_t)y * pitch + x0;
        float v[8];
        if (x0 + 8 <= W && (reinterpret_cast<uintptr_t>(src) & 15) == 0) {
            const float4 p = __ldg(reinterpret_cast<const float4 *>(src));
            const float4 q = __ldg(reinterpret_cast<const float4 *>(src + 4));
            v[0] = p.x; v[1] = p.y; v[2] = p.z; v[3] = p.w;
            v[4] = q.x; v[5] = q.y; v[6] = q.z; v[7] = q.w;
        } else {
#pragma unroll
            for (int t = 0; t < 8; ++t) v[t] = x0 + t < W ? __ldg(src + t) : c;   // c: 0 after - c
        }
#pragma unroll
        for (int t = 0; t < 8; ++t) v[t] = (v[t] - c) * sc;
        uint16_t *d = P + (int64_t)y * pq + x0;
        if (split) {
            uint32_t hw[4], lw[4];
#pragma unroll
            for (int t = 0; t < 4; ++t) b2split(v[2 * t], v[2 * t + 1], hw[t], lw[t]);
            *reinterpret_cast<uint4 *>(d) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
            *reinterpret_cast<uint4 *>(d + (int64_t)H * pq) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
        } else {
            *reinterpret_cast<uint4 *>(d) = make_uint4(h2pack(v[0], v[1]), h2pack(v[2], v[3]), h2pack(v[4], v[5]),
                                                       h2pack(v[6], v[7]));
        }
    }
}

__global__ void k_ones(const TcBankArgs a, const TcUnitDev *__restrict__ units, const TcFreqDev *__restrict__ freqs,
                       int nunits, float2 *__restrict__ A, float2 *__restrict__ B)
{
    // a programmatic dependent of k_minmax that does not read its result: it runs alongside,
    // and completes only after k_minmax has (so the kernels after it see both)
    pdl_launch_dependents();
    const int64_t n = (int64_t)nunits * (a.W + a.H);
    const int64_t gtid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x, gstride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = gtid; i < n; i += gstride) {
        const int u = (int)(i / (a.W + a.H)), p = (int)(i % (a.W + a.H));
        const bool is_x = p < a.W;
        const int pos = is_x ? p : p - a.W;
        const double2 v = ones_entry(a, freqs[units[u].s].R, u, is_x, pos, is_x ? a.W : a.H);
        const float2 f = make_float2((float)v.x, (float)v.y);
        if (is_x)
            A[(int64_t)u * a.W + pos] = f;
        else
            B[(int64_t)u * a.H + pos] = f;
    }
    pdl_wait();
    if (a.row_mt && a.corrA) {   // the centre is known now
        float c;
        int e;
        image_centre(a, c, e);
        corr_rows(a, units, freqs, nunits, a.W, a.H, c, a.corrA, a.corrB, gtid, gstride);
        if (a.p_tma) operand_image(a.img, a.pitch, a.H, a.W, c, e, a.pimg, a.pq, a.split, gtid, gstride);
    }
}

// Batch form of k_ones: grid (blocks, images), the tables of image blockIdx.y; then, once
// k_minmax_batch has completed, block 0 of every image reduces its partial keys into the
// image's (centre, exponent).
__global__ void k_ones_batch(const TcBankArgs a, const TcUnitDev *__restrict__ units,
                             const TcFreqDev *__restrict__ freqs, int nunits)
{
    pdl_launch_dependents();
    const TcImgDev im = a.imgs[blockIdx.y];
    const int64_t n = (int64_t)nunits * (im.W + im.H);
    const int64_t gtid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x, gstride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = gtid; i < n; i += gstride) {
        const int u = (int)(i / (im.W + im.H)), p = (int)(i % (im.W + im.H));
        const bool is_x = p < im.W;
        const int pos = is_x ? p : p - im.W;
        const double2 v = ones_entry(a, freqs[units[u].s].R, u, is_x, pos, is_x ? im.W : im.H);
        const float2 f = make_float2((float)v.x, (float)v.y);
        float2 *dst = const_cast<float2 *>(is_x ? im.onesA + (int64_t)u * im.W + pos : im.onesB + (int64_t)u * im.H + pos);
        *dst = f;
    }
    pdl_wait();
    // every block reduces the image's partial keys into its centre; block 0 records it
    __shared__ float cen_s;
    __shared__ int e_s;
    if (threadIdx.x < 32) {
        const unsigned *p = a.mm_part + (int64_t)blockIdx.y * kMmParts * 2;
        unsigned nlo = 0u, hik = 0u;
        for (int i = threadIdx.x; i < kMmParts; i += 32) {
            nlo = max(nlo, p[2 * i]);
            hik = max(hik, p[2 * i + 1]);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            nlo = max(nlo, __shfl_xor_sync(0xffffffffu, nlo, o));
            hik = max(hik, __shfl_xor_sync(0xffffffffu, hik, o));
        }
        if (threadIdx.x == 0) {
            float c;
            int e;
            centre_of(nlo, hik, c, e);
            cen_s = c;
            e_s = e;
            if (blockIdx.x == 0) a.img_ce[blockIdx.y] = make_float2(c, (float)e);
        }
    }
    __syncthreads();
    corr_rows(a, units, freqs, nunits, im.W, im.H, cen_s, im.corrA, im.corrB, gtid, gstride);
    if (a.p_tma) operand_image(im.img, im.pitch, im.H, im.W, cen_s, e_s, im.pimg, im.pq, a.split, gtid, gstride);
}

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
    g.smem_cols = col_stages(g.Kcol) ? 1024 + col_smem(g.Kcol, col_stages(g.Kcol)).total : (size_t)kSmemLimit + 1;
    return g;
}

size_t gabor_tc_smem_rows(int Kmax, int PWmax, int TY) { return 1024 + row_smem(Kmax, PWmax, TY).total; }
size_t gabor_tc_smem_cols(int Kmax) { return 1024 + col_smem(Kmax, col_stages(Kmax)).total; }

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

int gabor_tc_mt_tile_x() { return kMtTileX; }
int gabor_tc_mt_k(int R) { return round_up(kMtTileX + 2 * R, 64); }
int gabor_tc_mt_pw(int R) { return round_up(kMtTileX + 2 * R, 4); }
size_t gabor_tc_smem_rows_mt(int Kmax, int PWmax, int TY, int split)
{
    return 1024 + mt_smem(Kmax, PWmax, TY, split).total;
}
int gabor_tc_mt_tile_y(int Kmax, int PWmax, int split)
{
    return gabor_tc_smem_rows_mt(Kmax, PWmax, 64, split) <= (size_t)kSmemLimit ? 64 : 32;
}

int gabor_tc_mt_am_elems(int R, int split) { return (int)((split ? 2 : 1) * tstrip_bytes(gabor_tc_mt_k(R), 128) / 2); }
int gabor_tc_mt_gm_elems(int R, int col_ty, int split)
{
    return (int)((split ? 2 : 1) * tstrip_bytes(gabor_tc_geometry(R).Kcol, 2 * col_ty) / 2);
}

cudaError_t build_gabor_tc_gm(uint16_t *Gm, int R, double sigma, double ws, int col_ty, int split, cudaStream_t st)
{
    int e = 0;
    frexp(1.0 / (2.5066282746310002 * sigma), &e);
    const TcGeometry g = gabor_tc_geometry(R);
    const int nc = tstrip_cores(g.Kcol, 2 * col_ty);
    k_build_tstrip<<<(64 * nc + 255) / 256, 256, 0, st>>>(Gm, nc, col_ty - 1 + g.R8, R, sigma, ws, -e, split);
    return cudaGetLastError();
}

bool gabor_tc_mt_fits(int row_kmax, int row_pwmax, int col_kmax, int split)
{
    return gabor_tc_smem_rows_mt(row_kmax, row_pwmax, 32, split) <= (size_t)kSmemLimit &&
           1024 + mt_col_smem(col_kmax, 32, split, 1).total <= (uint32_t)kSmemLimit;
}

int gabor_tc_mt_col_ty(int col_kmax, int split)
{
    return 1024 + mt_col_smem(col_kmax, 64, split, 1).total <= (uint32_t)kSmemLimit ? 64 : 32;
}

// Operand stages of the modulated-tap column kernel: as many as fit, up to kMtColMaxStages.
int gabor_tc_mt_col_stages(int col_kmax, int col_ty, int split)
{
    int n = kMtColMaxStages;
    while (n > 1 && 1024 + mt_col_smem(col_kmax, col_ty, split, n).total > (uint32_t)kSmemLimit) --n;
    return n;
}

cudaError_t build_gabor_tc_am(uint16_t *Am, int R, double sigma, double wc, int split, cudaStream_t st)
{
    // the scale of the frequency's Toeplitz operands: |S(d) cos|, |S(d) sin| <= S(0)
    int e = 0;
    frexp(1.0 / (2.5066282746310002 * sigma), &e);
    const int nc = tstrip_cores(gabor_tc_mt_k(R), 128);
    k_build_tstrip<<<(64 * nc + 255) / 256, 256, 0, st>>>(Am, nc, kMtTileX - 1 + round_up(R, 8), R, sigma, wc, -e,
                                                            split);
    return cudaGetLastError();
}

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

cudaError_t build_gabor_tc_prefix(const double *unit_w, const TcUnitDev *units, const TcFreqDev *freqs,
                                  const double *sigma, int nunits, int stride, double2 *pre, cudaStream_t st)
{
    if (nunits == 0) return cudaSuccess;
    k_build_prefix<<<(2 * nunits + 63) / 64, 64, 0, st>>>(unit_w, units, freqs, sigma, nunits, stride, pre);
    return cudaGetLastError();
}

cudaError_t gabor_tc_prepare()
{
    cudaError_t e = cudaFuncSetAttribute(k_gabor_tc_rows, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemLimit);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_gabor_tc_rows_mt<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemLimit);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_gabor_tc_rows_mt<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemLimit);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_gabor_tc_cols_mt<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemLimit);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_gabor_tc_cols_mt<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemLimit);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_gabor_tc_cols, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemLimit);
    return e;
}

// Modulated-tap row-pass CTAs per SM: two when their shared memory fits (64 registers per
// thread, 128 TMEM columns each), so that one CTA's patch staging overlaps the other's MMAs and
// epilogue.
static int mt_rows_per_sm(size_t smem) { return 2 * (smem + 1024) <= (size_t)228 * 1024 ? 2 : 1; }

cudaError_t launch_gabor_tc(const TcBankArgs &a0, int sm_count, cudaStream_t st)
{
    TcBankArgs a = a0;
    a.col_nst = col_stages(a.col_kmax);
    if (a.col_nst < 2) return cudaErrorInvalidValue;
    if (a.row_mt && !gabor_tc_mt_fits(a.row_kmax, a.row_pwmax, a.col_kmax, a.split)) return cudaErrorInvalidValue;
    if (a.split && !a.row_mt) return cudaErrorInvalidValue;   // hi + lo operands: modulated-tap kernels only
    a.col_mt_nst = gabor_tc_mt_col_stages(a.col_kmax, a.col_mt_ty, a.split);
    const int n_row_items = a.nf * a.row_cnt, n_col_items = a.nf * a.col_cnt;
    const size_t smem_r = a.row_mt ? gabor_tc_smem_rows_mt(a.row_kmax, a.row_pwmax, a.row_ty, a.split)
                                   : gabor_tc_smem_rows(a.row_kmax, a.row_pwmax, a.row_ty);
    const size_t smem_c = a.row_mt ? 1024 + mt_col_smem(a.col_kmax, a.col_mt_ty, a.split, a.col_mt_nst).total
                                   : gabor_tc_smem_cols(a.col_kmax);
    cudaError_t e0 = cudaMemsetAsync(a.minmax, 0, 2 * sizeof(unsigned), st);
    if (e0 != cudaSuccess) return e0;
    const dim3 ag(std::max(1, std::min(4, (a.W + 255) / 256)), std::max(1, std::min(a.H, 2 * sm_count)));
    k_minmax<<<ag, 256, 0, st>>>(a.img, a.pitch, a.H, a.W, a.minmax);
    e0 = cudaGetLastError();
    if (e0 != cudaSuccess) return e0;
    {
        const int nu = a.nf * a.nu_f;
        // threads for the tables, or for the operand image (8 columns each)
        const int64_t n = std::max<int64_t>((int64_t)nu * (a.W + a.H), a.p_tma ? (int64_t)a.H * ((a.W + 7) / 8) : 0);
        const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 4 * sm_count));
        e0 = launch_pdl(k_ones, dim3(blocks), dim3(256), 0, st, a, a.units, a.freqs, nu,
                        const_cast<float2 *>(a.onesA), const_cast<float2 *>(a.onesB));
        if (e0 != cudaSuccess) return e0;
    }
    if (n_row_items > 0) {
        cudaError_t e;
        if (a.row_mt) {
            e = launch_pdl(a.split ? k_gabor_tc_rows_mt<true> : k_gabor_tc_rows_mt<false>,
                           dim3(std::min(n_row_items, sm_count * mt_rows_per_sm(smem_r))), dim3(512), smem_r, st, a);
        } else {
            k_gabor_tc_rows<<<std::min(n_row_items, sm_count), 512, smem_r, st>>>(a);
            e = cudaGetLastError();
        }
        if (e != cudaSuccess) return e;
    }
    if (n_col_items > 0) {
        if (a.row_mt)
            return launch_pdl(a.split ? k_gabor_tc_cols_mt<true> : k_gabor_tc_cols_mt<false>,
                              dim3(std::min(n_col_items, sm_count)), dim3(kMtColThreads), smem_c, st, a);
        else
            k_gabor_tc_cols<<<std::min(n_col_items, sm_count), kColThreads, smem_c, st>>>(a);
        return cudaGetLastError();
    }
    return cudaSuccess;
}

cudaError_t launch_gabor_tc_batch(const TcBankArgs &a0, int sm_count, cudaStream_t st)
{
    TcBankArgs a = a0;
    if (!a.imgs || !a.row_mt || !gabor_tc_mt_fits(a.row_kmax, a.row_pwmax, a.col_kmax, a.split))
        return cudaErrorInvalidValue;
    a.col_nst = col_stages(a.col_kmax);
    a.col_mt_nst = gabor_tc_mt_col_stages(a.col_kmax, a.col_mt_ty, a.split);
    const size_t smem_r = gabor_tc_smem_rows_mt(a.row_kmax, a.row_pwmax, a.row_ty, a.split);
    const size_t smem_c = 1024 + mt_col_smem(a.col_kmax, a.col_mt_ty, a.split, a.col_mt_nst).total;
    static_assert(kMmParts == 64, "k_minmax_batch runs 8 x 8 blocks per image");
    k_minmax_batch<<<dim3(8, 8, a.nimg), 256, 0, st>>>(a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    e = launch_pdl(k_ones_batch, dim3(16, a.nimg), dim3(256), 0, st, a, a.units, a.freqs, a.nf * a.nu_f);
    if (e != cudaSuccess) return e;
    if (a.n_row > 0) {
        e = launch_pdl(a.split ? k_gabor_tc_rows_mt<true> : k_gabor_tc_rows_mt<false>,
                       dim3(std::min(a.n_row, sm_count * mt_rows_per_sm(smem_r))), dim3(512), smem_r, st, a);
        if (e != cudaSuccess) return e;
    }
    if (a.n_col > 0)
        e = launch_pdl(a.split ? k_gabor_tc_cols_mt<true> : k_gabor_tc_cols_mt<false>, dim3(std::min(a.n_col, sm_count)),
                       dim3(kMtColThreads), smem_c, st, a);
    return e;
}

}  // namespace gb
