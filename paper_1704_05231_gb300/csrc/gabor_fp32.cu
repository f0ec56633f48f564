// Fused FP32 Gabor filter-bank kernel (K1 + K2): Algorithm 1 of arXiv 1704.05231 for every
// frequency and orientation of a plan, on FP32 CUDA cores, in one launch.
//
// A CTA owns one work item: one horizontal pass ("unit": orientation theta_a at frequency
// omega_s and, when present, its mirror pi - theta_a), one strip of 32 image columns and one
// segment of rows.  Work items are sorted by cost, largest first.  The CTA walks down its
// segment in chunks of TH rows:
//
//   row pass  (Eq. 5-6)   rows of f (strip plus an R-wide halo) arrive by cp.async into a
//                         double buffer, one row block ahead of use, and become
//                             J_theta(x) = sum_d S(d) f(x + d) exp(-i omega^c d)
//                         in one of two forms: demodulate by (cos, sin)(omega^c k), smooth
//                         with the real Gaussian S, remodulate (Eq. 5-6 step by step), or one
//                         pass with the modulated taps S(d) exp(-i omega^c d), the same sum
//                         without the demodulated copy of the rows (default: half the
//                         shared-memory traffic).  J is immediately demodulated by
//                         (cos, sin)(omega^s y) into the column signals of Eq. 10:
//                             f_cr + f_si, f_sr - f_ci            (theta_a,      Eq. 7-9)
//                             f_cr - f_si, f_sr + f_ci            (pi - theta_a, Eq. 15-16)
//                         which go into a ring buffer of rows in shared memory.  J never
//                         leaves the chip; J_{pi-theta} = J*_theta (Eq. 13) costs nothing.
//   column pass (Eq. 7-9) smooth the ring's signals along y with S, remodulate by
//                         (cos, sin)(omega^s y) and store F_theta_a (and F_{pi-theta_a}).
//
// The ring keeps the 2R rows of vertical halo between chunks, so every row's horizontal pass
// is computed once per segment (plus 2R rows of prologue per segment).
#include <algorithm>

#include "internal.h"
#include "conv_fp32.cuh"
#include "tc_common.cuh"

namespace gb {

namespace {

struct Smem {
    float2 *ring2;   // ring of column signals: [RS][33] float2 per plane; paired units keep
                     // (P, Q) of theta_a in plane 0 and (P', Q') of pi - theta_a in plane 1
    float2 *stage;   // demodulation form: TH x SW demodulated rows (f_c, f_s)
    float *raw;      // two buffers of TH x RW floats
    float2 *ctaps;   // modulated taps: 2 x (Tpad + 8) complex taps S(t - R) exp(-i omega^c (t - R))
    float2 *phx;     // demodulation form: SW + 1 row phases
    float *taps;     // Tpad + 8 real taps (column pass)
    uint64_t *bars;  // pipelined schedule: full[2], empty[2]; TMA row loads: full[2]; then the
                     // abort flag
};

// modulated taps: one set per unit of a (twin) item
__host__ __device__ __forceinline__ int ctap_count(const FreqDev &f) { return f.mtaps ? 2 * (f.Tpr + 8) : 0; }
__host__ __device__ __forceinline__ int phx_count(const FreqDev &f) { return f.mtaps ? 0 : f.SW + 1; }

// Every region starts on a 16-byte boundary (RS, TH multiples of 8; SW odd; Tpad + 8 even).
// ALIGN (kernels with TMA row loads): the base on a 128-byte boundary, and so the raw buffers
// under modulated taps (SW = 0, ring rows of 33 float2 pairs, RS and TH multiples of 8, RW a
// multiple of 4), as TMA writes want.
template <bool ALIGN>
__device__ __forceinline__ Smem carve(unsigned char *base0, const FreqDev &f)
{
    unsigned char *base =
        ALIGN ? reinterpret_cast<unsigned char *>(((uintptr_t)base0 + 127) & ~(uintptr_t)127) : base0;
    Smem s;
    s.ring2 = reinterpret_cast<float2 *>(base);
    s.stage = s.ring2 + (size_t)2 * f.RS * (kStripW + 1);
    s.raw = reinterpret_cast<float *>(s.stage + (size_t)f.TH * f.SW);
    s.ctaps = reinterpret_cast<float2 *>(s.raw + (size_t)2 * f.TH * f.RW);
    s.phx = s.ctaps + ctap_count(f);
    s.taps = reinterpret_cast<float *>(s.phx + phx_count(f));
    s.bars = reinterpret_cast<uint64_t *>(((uintptr_t)(s.taps + f.Tpad + 8) + 7) & ~(uintptr_t)7);
    return s;
}

}  // namespace

size_t gabor_fp32_smem_bytes(const FreqDev &f)
{
    return (size_t)f.RS * (kStripW + 1) * sizeof(float4) + (size_t)f.TH * f.SW * sizeof(float2) +
           (size_t)2 * f.TH * f.RW * sizeof(float) + (size_t)(ctap_count(f) + phx_count(f)) * sizeof(float2) +
           (size_t)(f.Tpad + 8) * sizeof(float) + 8 + 4 * sizeof(uint64_t) + 16 + 128;
}

// Dynamic shared memory one CTA may take when `ctas` CTAs share an SM (228 KB per SM, 1 KB
// of it reserved per CTA, and the kernel's own static word).
size_t gabor_fp32_smem_budget(int ctas)
{
    return (size_t)(kSmemPerSm - ctas * kSmemCtaReserve) / ctas - kStaticSmemReserve;
}

FreqDev gabor_fp32_geometry(int R, int tile_rows, bool pipelined, bool mtaps, int ctas)
{
    FreqDev f{};
    f.R = R;
    f.T = 2 * R + 1;
    f.Tpad = round_up(f.T, 8);
    f.mtaps = mtaps ? 1 : 0;
    f.Rw = mtaps ? round_up(R, 4) : R;
    f.Tr = f.Rw + R + 1;
    f.Tpr = round_up(f.Tr, 8);
    if (mtaps) {
        // no demodulated copy; raw rows hold the whole tap window of every output (zeros past
        // the halo) and are = 4 (mod 32) floats apart, so that the 16-byte window loads of the
        // 8 lanes (8 rows) of a quarter warp fall on distinct banks
        f.SW = 0;
        f.RW = round_up(kStripW + f.Tpr - 1, 32) + 4;
    } else {
        f.SW = stage_width(kStripW + f.Tpad);
        f.RW = round_up(kStripW + f.T - 1, 4);
    }
    // the pipelined schedule takes 32 rows per chunk at most, and its ring holds two chunks
    int TH = tile_rows > 0 ? tile_rows : (pipelined ? 32 : 64);
    if (pipelined) TH = std::min(TH, 32);
    for (;;) {
        f.TH = TH;
        f.RS = round_up((pipelined ? 2 * TH : TH) + f.T - 1, 8);
        if (gabor_fp32_smem_bytes(f) <= gabor_fp32_smem_budget(ctas) || TH <= 8) break;
        TH /= 2;
    }
    return f;
}

// Offset of output (plane p, row 0, column x): plane-major out[p][y][x] or pixel-major
// out[y][x][p] (the n_freq x n_theta feature vector of a pixel contiguous).
__device__ __forceinline__ int64_t out_offset(const BankArgs &a, int p, int64_t plane, int x)
{
    return a.layout ? (int64_t)x * a.nplanes + p : (int64_t)p * plane + x;
}

// NW = 16: one CTA of 16 warps per SM; NW = 8: two CTAs of 8 warps per SM, whose phases
// (row pass, barrier, column pass, epilogues) interleave on the SM.

// PIPE = false: all 16 warps run the phases of a chunk in turn (row pass, then column pass).
// PIPE = true: warps 0-7 run the row passes, warps 8-15 the column passes, one chunk apart;
// the ring holds two chunks and mbarriers hand chunks over (bounded waits).  Returns false
// when a wait gave up (the status word is set).  NW warps per CTA (PIPE: 16).  MT: row pass
// with modulated taps; an item
// of this form may also carry two unpaired units of one frequency ("twins"): two row passes
// into the two ring planes, whose column passes then fill both halves of the CTA.
// RT: the instance with TMA row loads (one-image launches under the zero rule); the others
// carry none of its code.
template <bool PIPE, bool MT, int NW, bool RT>
__device__ __forceinline__ bool gabor_fp32_item(const BankArgs &a, const WorkItem it, unsigned char *smem_raw)
{
    const UnitDev u = a.units[it.unit];
    const FreqDev f = a.freqs[u.s];
    const ImageDev im = a.imgs ? a.imgs[it.img] : a.img0;
    const bool paired = u.plane_b >= 0;
    const int utw = MT ? u.twin : -1;
    const bool twin = utw >= 0;
    const UnitDev u2 = a.units[twin ? utw : it.unit];   // the second unit of a twin item
    const bool two = paired || twin;                     // two ring planes
    const int x0 = it.strip * kStripW;
    const int ys = it.y0, ye = it.y1;
    const int tid = threadIdx.x;
    const int warp = tid >> 5, lane = tid & 31;
    const int stride = kStripW + 1;
    const int R = f.R, TH = f.TH, RS = f.RS, SW = f.SW, RW = f.RW;
    const int Rw = f.Rw;
    const int ncols = kStripW + f.Tr - 1;       // input columns x0 - Rw .. x0 + 31 + R
    // full 8-tap chunks, and one tail tap for filters of 8 k + 1 taps (R = 0 mod 4) instead of
    // a chunk of 7 zero taps; the row pass runs over its Tr taps, the column pass over T
    const bool tail1 = (f.T & 7) == 1;
    const int nchunks = tail1 ? f.T / 8 : f.Tpad / 8;
    const bool tail1r = (f.Tr & 7) == 1;
    const int nchunks_r = tail1r ? f.Tr / 8 : f.Tpr / 8;
    const int64_t plane = (int64_t)im.H * im.W;
    const int64_t ystride = a.layout ? (int64_t)im.W * a.nplanes : (int64_t)im.W;   // between output rows
    const Smem sm = carve<RT>(smem_raw, f);
    const float4 *taps4 = reinterpret_cast<const float4 *>(sm.taps);
    const float4 *ctaps4 = reinterpret_cast<const float4 *>(sm.ctaps);
    static_assert(NW == 16 || (NW == 8 && !PIPE), "16 warps, or 8 without the pipelined schedule");
    constexpr int kThreadsCta = 32 * NW;
    constexpr int kRowWarps = PIPE ? 8 : NW;   // warps that load rows and run the row pass
    constexpr int kRB = kRowWarps / 2;         // 8-row blocks of one row-pass sweep
    auto sync_rows = [&]() {
        if (PIPE)
            named_barrier(1, kRowWarps * 32);
        else
            __syncthreads();
    };

    uint64_t *full = sm.bars, *empty = sm.bars + 2;   // pipelined hand-over, per ring half
    volatile int *abort_s = reinterpret_cast<volatile int *>(sm.bars + 4);
    // row blocks by TMA: boxes of RW columns from x0 - Rw (a multiple of 4 floats, 16 bytes, as a
    // tiled copy needs) x TH rows, zeros outside the image; completion on sm.bars[b & 1]
    const bool rtma = RT && !PIPE && MT && a.imgs == nullptr && ((a.raw_mask >> u.s) & 1u);
    if (rtma) {
        if (tid == 0) {
            mbar_init(&sm.bars[0], 1);
            mbar_init(&sm.bars[1], 1);
            *abort_s = 0;
            mbar_fence_init();
        }
        __syncthreads();
    }
    if (PIPE && tid == 0) {
        mbar_init(&full[0], kRowWarps * 32);
        mbar_init(&full[1], kRowWarps * 32);
        mbar_init(&empty[0], (NW - kRowWarps) * 32);
        mbar_init(&empty[1], (NW - kRowWarps) * 32);
        *abort_s = 0;
        mbar_fence_init();
    }
    for (int i = tid; i < f.Tpad + 8; i += kThreadsCta) sm.taps[i] = i < f.Tpad ? f.taps[i] : 0.f;
    const bool ext = a.bmode != kBoundaryZero;
    if (MT) {
        // taps S(d) exp(-i omega^c d), d = t - Rw: (cos, -sin) from the unit's phase table,
        // zero for |d| > R (a twin item: both units' taps, one set after the other)
        for (int i = tid; i < (twin ? 2 : 1) * (f.Tpr + 8); i += kThreadsCta) {
            const int t = i % (f.Tpr + 8) - (Rw - R);   // index into the T taps S(t - R)
            const bool in = t >= 0 && t < f.T;
            const float2 ph = in ? (i < f.Tpr + 8 ? u.phx : u2.phx)[t - R] : make_float2(0.f, 0.f);
            const float g = in ? f.taps[t] : 0.f;
            sm.ctaps[i] = make_float2(g * ph.x, -(g * ph.y));
        }
        // raw columns past the halo are read (by zero taps) and never copied: zero them (the
        // TMA boxes cover them)
        const int tail = RW - ncols;
        if (!rtma)
            for (int i = tid; i < 2 * TH * tail; i += kThreadsCta) sm.raw[(size_t)(i / tail) * RW + ncols + i % tail] = 0.f;
    } else {
        // Demodulation phases at the staged positions (beyond the image only for non-zero
        // rules, whose extended samples are demodulated at their own positions).
        for (int j = tid; j <= SW; j += kThreadsCta) {
            const int gx = x0 - R + j;
            sm.phx[j] = (j < ncols && (ext || (gx >= 0 && gx < im.W))) ? u.phx[gx] : make_float2(0.f, 0.f);
        }
    }
    for (int i = tid; i < 2 * RS * stride; i += kThreadsCta) sm.ring2[i] = make_float2(0.f, 0.f);

    // Row blocks: the prologue [ys - R, need_0) in pieces of TH rows, then one block per
    // later chunk k covering [need_{k-1}, need_k), need_k = min(ys + (k+1) TH, ye) + R.
    const int ring_origin = ys - R;
    const int need0 = min(ys + TH, ye) + R;
    const int npro = (need0 - ring_origin + TH - 1) / TH;
    const int nch = (ye - ys + TH - 1) / TH;
    const int nblocks = npro + nch - 1;
    auto block_rows = [&](int b, int &start, int &n) {
        if (b < npro) {
            start = ring_origin + b * TH;
            n = min(TH, need0 - start);
        } else {
            const int k = b - npro + 1;
            start = min(ys + k * TH, ye) + R;
            n = min(ys + (k + 1) * TH, ye) + R - start;
        }
    };
    // Issue the async copy of row block b into raw buffer b & 1 (zeros outside the image).
    auto issue = [&](int b) {
        int start, n;
        block_rows(b, start, n);
        float *dst = sm.raw + (size_t)(b & 1) * TH * RW;
        if (rtma) {
            if (tid == 0) {
                fence_proxy_async_smem();   // the generic reads of this buffer's last block precede the copy
                mbar_arrive_expect_tx(&sm.bars[b & 1], (uint32_t)TH * RW * 4u);
                tma_load_2d(smem_u32(dst), &a.raw_map[u.s], x0 - Rw, start, &sm.bars[b & 1]);
            }
            return;
        }
        if (!ext) {
            // strips whose window lies inside the image: 16-byte copies for rows that start on
            // a 16-byte boundary (raw rows do: RW and x0 - Rw are multiples of 4 under
            // modulated taps), the last ncols mod 4 columns by 4-byte copies
            const bool xin = MT && x0 - Rw >= 0 && x0 - Rw + ncols <= im.W;
            const int n16 = ncols >> 2;
            for (int r = warp; r < n; r += kRowWarps) {
                const int y = start + r;
                const bool yin = y >= 0 && y < im.H;
                float *d = dst + (size_t)r * RW;
                const float *src = im.img + (int64_t)(yin ? y : 0) * im.pitch;
                if (yin && xin && (reinterpret_cast<uintptr_t>(src + (x0 - Rw)) & 15) == 0) {
                    const float *s0 = src + (x0 - Rw);
                    for (int j = lane; j < n16; j += 32) cp_async16(d + 4 * j, s0 + 4 * j);
                    for (int j = 4 * n16 + lane; j < ncols; j += 32) cp_async4(d + j, s0 + j, 4);
                } else {
                    for (int j = lane; j < ncols; j += 32) {
                        const int gx = x0 - Rw + j;
                        const bool ok = yin && gx >= 0 && gx < im.W;
                        cp_async4(d + j, ok ? (const void *)(src + gx) : (const void *)im.img, ok ? 4 : 0);
                    }
                }
            }
        } else {
            for (int r = warp; r < n; r += kRowWarps) {
                const float *src = im.img + (int64_t)ext_coord(start + r, im.H, a.bmode) * im.pitch;
                for (int j = lane; j < ncols; j += 32)
                    cp_async4(dst + (size_t)r * RW + j, src + ext_coord(x0 - Rw + j, im.W, a.bmode), 4);
            }
        }
        cp_async_commit();
    };

    // Horizontal pass of row block b (raw data already waited for).
    auto row_pass = [&](int b) {
        int start, n;
        block_rows(b, start, n);
        const float *rawb = sm.raw + (size_t)(b & 1) * TH * RW;
        if (!MT) {
            // demodulation f_c, f_s of Eq. 5 into the float2 stage: a lane keeps the phase of
            // its column and demodulates the warp's rows (at most 4), all loads issued first
            constexpr int kRowsPerWarp = 64 / kRowWarps;   // TH <= 64
            for (int j = lane; j < SW; j += 32) {
                const float2 ph = sm.phx[j];
                float v[kRowsPerWarp];
#pragma unroll
                for (int i = 0; i < kRowsPerWarp; ++i) {
                    const int r = warp + i * kRowWarps;
                    v[i] = (r < n && j < ncols) ? rawb[(size_t)r * RW + j] : 0.f;
                }
#pragma unroll
                for (int i = 0; i < kRowsPerWarp; ++i) {
                    const int r = warp + i * kRowWarps;
                    if (r < n) sm.stage[(size_t)r * SW + j] = make_float2(v[i] * ph.x, v[i] * ph.y);
                }
            }
            sync_rows();
        }
        // 16 (row, 8-column group) outputs per warp, sweeps of 8 kRB rows x 4 groups; the two
        // half warps take the two halves of the tap chunks and add them with one shuffle.
        // Demodulation form: a half warp covers 8 rows x groups 2 q0, 2 q0 + 1 (distinct bank
        // pairs of the float2 stage).  Modulated taps (raw rows 4 mod 32 floats apart, window
        // loads of 16 bytes): each quarter warp reads 8 different rows, which fall on distinct
        // banks whatever the group and tap half.
        const int hl = lane & 15, half = lane >> 4;
        const int q0 = warp / kRB;
        int nh = (nchunks_r + 1) >> 1;
        if (MT && (nh & 3) == 0 && (nchunks_r & 1)) --nh;   // same longest half, odd split
        const int q = MT ? ((nh & 3) == 2 ? 2 * q0 + (hl >> 3) : q0 + 2 * (hl >> 3)) : (hl >> 3) | (q0 << 1);
        for (int r0 = 0; r0 < n; r0 += 8 * kRB) {
        const int r = r0 + ((hl & 7) | ((warp % kRB) << 3));
        // Warp-uniform: the warp's 8 rows start inside the block (rows < TH, so every stage read
        // is in bounds); rows r >= n are computed but not stored.
        if (r0 + 8 * (warp % kRB) < n) {
            const int c0 = half ? nh : 0, cnt = half ? nchunks_r - nh : nh;
            const int y = start + r;
            const int base = ((y - ring_origin) % RS) * stride + 8 * q;
            const bool yin = ext || (y >= 0 && y < im.H);
#pragma unroll 1
            for (int v = 0; v < (twin ? 2 : 1); ++v) {   // the unit, then its twin
                // the row's phase, loaded before the convolution so that its latency is hidden
                const float2 cy = yin ? (v ? u2.phy : u.phy)[y] : make_float2(0.f, 0.f);
                float2 acc[8];
#pragma unroll
                for (int j = 0; j < 8; ++j) acc[j] = make_float2(0.f, 0.f);
                // the tail tap goes to the half warp that ends at the last chunk
                if (MT)
                    conv8_linear_ct4(rawb + (size_t)r * RW + 8 * q + 8 * c0,
                                     ctaps4 + v * ((f.Tpr + 8) / 2) + 4 * c0, cnt, acc, tail1r && half);
                else
                    conv8_linear<float2>(sm.stage + (size_t)r * SW + 8 * q + 8 * c0, taps4 + 2 * c0, cnt, acc,
                                         tail1r && half);
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    acc[j].x += __shfl_xor_sync(0xffffffffu, acc[j].x, 16);
                    acc[j].y += __shfl_xor_sync(0xffffffffu, acc[j].y, 16);
                }
                float2 *ring = sm.ring2 + (size_t)v * RS * stride + base;
#pragma unroll
                for (int jj = 0; jj < 4; ++jj) {
                    if (r >= n) break;
                    const int j = jj + 4 * half;   // each half warp finishes 4 of the 8 outputs
                    const float2 aj = half ? acc[jj + 4] : acc[jj];
                    float jr, ji;
                    if (MT) {
                        jr = aj.x;
                        ji = aj.y;
                    } else {
                        const float2 px = sm.phx[R + 8 * q + j];
                        const float A = aj.x, B = aj.y;
                        // Eq. 5-6: Re J = cos A + sin B, Im J = sin A - cos B
                        jr = fmaf(px.x, A, px.y * B);
                        ji = fmaf(px.y, A, -px.x * B);
                    }
                    // Eq. 10: f_cr, f_sr, f_ci, f_si
                    const float fcr = jr * cy.x, fsr = jr * cy.y, fci = ji * cy.x, fsi = ji * cy.y;
                    ring[j] = make_float2(fcr + fsi, fsr - fci);
                    if (paired) sm.ring2[(size_t)RS * stride + base + j] = make_float2(fcr - fsi, fsr + fci);
                }
            }
        }
        }
    };

    // Vertical pass for output rows [c, c + nout).
    // Two planes: one half of the column warps smooths plane 0 ((P, Q) of theta_a), the other
    // plane 1 ((P', Q') of pi - theta_a, or the twin's (P, Q)), 8 rows per warp at a time; a
    // single unpaired unit uses all column warps on rows.
    auto col_pass = [&](int c, int nout) {
        const int cw = PIPE ? warp - 8 : warp;          // column-warp index
        const int ncw = PIPE ? 8 : NW;
        const int xl = lane;
        const int sub = two ? cw / (ncw / 2) : 0;
        const int ybase = 8 * (two ? cw % (ncw / 2) : cw);
        const int ystep = 8 * (two ? ncw / 2 : ncw);
        const int x = x0 + xl;
        const float2 *phy = (sub && twin) ? u2.phy : u.phy;
        const int oplane = sub ? (twin ? u2.plane_a : u.plane_b) : u.plane_a;
        for (int yb = ybase; yb < nout; yb += ystep) {
            const int slot0 = (c - ys + yb) % RS;
            // the 8 rows' phases, loaded before the convolution so that their latency is hidden
            const int jn = nout - yb;
            const float2 *py = phy + (c + yb);
            float2 cyv[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) cyv[j] = j < jn ? py[j] : make_float2(0.f, 0.f);
            float2 acc[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) acc[j] = make_float2(0.f, 0.f);
            conv8_ring<float2, kStripW + 1>(sm.ring2 + (size_t)sub * RS * stride + xl, RS, slot0, taps4, nchunks, acc,
                                            tail1);
            if (x < im.W) {
                // output row c + yb + j: one pointer stepped by the row stride
                float2 *o = im.out + out_offset(a, oplane, plane, x) + (int64_t)(c + yb) * ystride;
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    if (j < jn) {
                        const float2 cy = cyv[j];
                        const float P = acc[j].x, Q = acc[j].y;
                        // Eq. 7-8 (theta_a) or Eq. 15-16 (pi - theta_a)
                        __stcs(o, make_float2(fmaf(cy.x, P, cy.y * Q), fmaf(cy.y, P, -cy.x * Q)));
                    }
                    o += ystride;
                }
            }
        }
    };

    // Make row block b visible with block b + 1 in flight, then run the row pass of block b.
    // The demodulation form reads the raw buffer before its own barrier, so block b + 1 can
    // be issued before it; the modulated-tap form reads raw rows until the end of its pass, so
    // block b + 1 (which refills the buffer of block b - 1) is issued after the barrier.
    // Returns false when a TMA wait gave up (every thread of the CTA alike).
    auto advance = [&](int b) -> bool {
        if (rtma) {
            const bool ok = mbar_wait(&sm.bars[b & 1], (b >> 1) & 1, abort_s);
            if (__syncthreads_or(!ok)) {   // raw block b landed everywhere, or a wait gave up
                if (tid == 0) {
                    // the copy of block b lands before the CTA moves on; report the stop
                    volatile int dummy = 0;
                    mbar_wait(&sm.bars[b & 1], (b >> 1) & 1, &dummy);
                    if (a.status) atomicExch(a.status, 33);
                }
                return false;
            }
            if (b + 1 < nblocks) issue(b + 1);
        } else if (MT) {
            cp_async_wait<0>();
            sync_rows();   // raw block b visible; the row pass of block b - 1 is done
            if (b + 1 < nblocks) issue(b + 1);
        } else {
            if (b + 1 < nblocks) {
                issue(b + 1);
                cp_async_wait<1>();
            } else {
                cp_async_wait<0>();
            }
            sync_rows();   // raw block b visible; previous stage / ring readers done
        }
        row_pass(b);
        return true;
    };

    if (!PIPE) {
        issue(0);
        int b = 0;
        for (int k = 0; k < nch; ++k) {
            const int last = (k == 0) ? npro : npro + k;   // blocks [b, last) feed chunk k
            for (; b < last; ++b)
                if (!advance(b)) return false;
            __syncthreads();       // ring rows of chunk k complete
            const int c = ys + k * TH;
            col_pass(c, min(TH, ye - c));
        }
        return true;
    }
    // ---- pipelined: chunk k's rows (warps 0-7) overlap chunk k-1's column pass (warps 8-15)
    __syncthreads();   // taps, phases, zeroed ring and barriers visible to both groups
    bool ok = true;
    if (warp < kRowWarps) {
        issue(0);
        int b = 0;
        for (int k = 0; k < nch; ++k) {
            // chunk k's rows reuse the ring slots of chunk k-2's window
            const bool failed = k >= 2 && !mbar_wait(&empty[k & 1], ((k - 2) >> 1) & 1, abort_s);
            if (named_barrier_or(1, kRowWarps * 32, failed)) {
                ok = false;
                break;
            }
            const int last = (k == 0) ? npro : npro + k;
            for (; b < last; ++b) advance(b);   // async copies: never gives up
            mbar_arrive(&full[k & 1]);   // this thread's ring rows of chunk k are written
        }
        cp_async_wait<0>();
    } else {
        for (int k = 0; k < nch; ++k) {
            if (!mbar_wait(&full[k & 1], (k >> 1) & 1, abort_s)) {
                ok = false;
                break;
            }
            const int c = ys + k * TH;
            col_pass(c, min(TH, ye - c));
            mbar_arrive(&empty[k & 1]);
        }
    }
    if (!ok && lane == 0) {
        *abort_s = 1;
        if (a.status) atomicExch(a.status, 35);
    }
    return ok;
}

// Work item `item` of a single-image launch, decoded from the groups (uniform per CTA).
__device__ __forceinline__ WorkItem decode_item(const BankArgs &a, int item)
{
    int g = 0;
    while (g + 1 < a.ngroups && item >= a.groups[g + 1].first) ++g;
    const ItemGroup &G = a.groups[g];
    const int local = item - G.first;
    const int seg = local % G.nseg, rest = local / G.nseg;
    const int y0 = seg * G.seg_len;
    return WorkItem{0, G.u0 + G.ustride * (rest / G.nstrips), rest % G.nstrips, y0, min(a.img0.H, y0 + G.seg_len)};
}

// Persistent CTAs pull work items (cost-sorted, largest first) from a device counter that the
// launcher zeroes before the launch.
// A CTA stops taking items after a bounded wait gave up (pipelined schedule).
template <bool PIPE, bool MT, int NW, bool RT>
__global__ void __launch_bounds__(32 * NW, 16 / NW) k_gabor_fp32(const __grid_constant__ BankArgs a)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int next_item;
    for (;;) {
        if (threadIdx.x == 0) next_item = atomicAdd(a.counter, 1);
        __syncthreads();
        const int item = next_item;
        if (item >= a.nitems) break;
        const WorkItem it = a.items ? a.items[item] : decode_item(a, item);
        const bool ok = gabor_fp32_item<PIPE, MT, NW, RT>(a, it, smem_raw);
        // shared memory is reused by the next item
        const bool failed = __syncthreads_or(!ok);
        if (PIPE && threadIdx.x == 0) {
            const FreqDev &f = a.freqs[a.units[it.unit].s];
            uint64_t *bars = carve<RT>(smem_raw, f).bars;
            for (int i = 0; i < 4; ++i) mbar_inval(bars + i);
        }
        if (RT && !PIPE && MT && threadIdx.x == 0) {
            const int s = a.units[it.unit].s;
            if ((a.raw_mask >> s) & 1u) {
                uint64_t *bars = carve<RT>(smem_raw, a.freqs[s]).bars;
                for (int i = 0; i < 2; ++i) mbar_inval(bars + i);
            }
        }
        if (failed) break;
    }
}

template <bool PIPE, bool MT, int NW, bool RT = false>
cudaError_t prepare_one()
{
    // the kernel's own static shared memory (the work-queue word) counts against the limit
    return cudaFuncSetAttribute(k_gabor_fp32<PIPE, MT, NW, RT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                kSmemLimit - kStaticSmemReserve);
}

cudaError_t gabor_fp32_prepare()
{
    cudaError_t e = prepare_one<false, false, 16>();
    if (e == cudaSuccess) e = prepare_one<false, true, 16>();
    if (e == cudaSuccess) e = prepare_one<true, false, 16>();
    if (e == cudaSuccess) e = prepare_one<true, true, 16>();
    if (e == cudaSuccess) e = prepare_one<false, false, 8>();
    if (e == cudaSuccess) e = prepare_one<false, true, 8>();
    if (e == cudaSuccess) e = prepare_one<false, true, 16, true>();
    if (e == cudaSuccess) e = prepare_one<false, true, 8, true>();
    return e;
}

template <bool PIPE, bool MT, int NW, bool RT = false>
cudaError_t launch_one(const BankArgs &a, int nitems, size_t smem, int sm_count, cudaStream_t st)
{
    int cps = 1;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&cps, k_gabor_fp32<PIPE, MT, NW, RT>, 32 * NW, smem);
    if (e != cudaSuccess) return e;
    const int grid = std::min(nitems, std::max(1, cps) * sm_count);
    k_gabor_fp32<PIPE, MT, NW, RT><<<grid, 32 * NW, smem, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_gabor_fp32(const BankArgs &a0, int nitems, size_t smem, int sm_count, cudaStream_t st)
{
    if (nitems <= 0) return cudaSuccess;
    BankArgs a = a0;
    a.nitems = nitems;
    cudaError_t e = cudaMemsetAsync(a.counter, 0, sizeof(int), st);
    if (e != cudaSuccess) return e;
    if (a.pipelined)
        return a.mtaps ? launch_one<true, true, 16>(a, nitems, smem, sm_count, st)
                       : launch_one<true, false, 16>(a, nitems, smem, sm_count, st);
    const bool rt = a.mtaps && a.raw_mask != 0 && a.imgs == nullptr;   // TMA row loads somewhere
    if (a.ctas == 2) {
        if (rt) return launch_one<false, true, 8, true>(a, nitems, smem, sm_count, st);
        return a.mtaps ? launch_one<false, true, 8>(a, nitems, smem, sm_count, st)
                       : launch_one<false, false, 8>(a, nitems, smem, sm_count, st);
    }
    if (rt) return launch_one<false, true, 16, true>(a, nitems, smem, sm_count, st);
    return a.mtaps ? launch_one<false, true, 16>(a, nitems, smem, sm_count, st)
                   : launch_one<false, false, 16>(a, nitems, smem, sm_count, st);
}

}  // namespace gb
